// Batches of DDI evaluations and the spread-tile autotuner.
//
// A batch holds one plan per density (each with its own grid, box, dipole axes and
// quadrature, Sec. 2.1) and evaluates Phi_i = U_dip,i * rho_i for all of them in one
// call.  The plans are independent (private fine grids, node arrays and work lists), so
// the batch spreads them over a few side streams, largest first onto the least loaded
// stream, joined back to the caller's stream by events.  With DDI_BATCH_GRAPH the whole
// fork/join of launches is recorded once into a CUDA graph and every later call with the
// same pointers replays it with one cudaGraphLaunch; new pointers re-record it and update
// the executable graph in place.
//
// The autotuner picks the spread tile of a plan by timing the spread (with its
// partial-plane reduction) for a list of candidate tiles on the plan's own node set and
// keeping the fastest; for column plans it picks the visits per work unit, and for 2D
// plans with the automatic scheme it times both schemes and keeps the faster.  The node positions on the fine grid depend only on the grid, the
// quadrature sizes and kmax h, not on the box length or the dipole axes, so the result
// is cached per such shape (and device) for the life of the process.
#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>

#include "common.cuh"

namespace ddi {
namespace {

std::mutex g_tune_mu;
struct TuneResult {
  std::array<int, 3> tile;
  int chunk;  // column plans: visits per work unit
  double ms;
  int kind;   // the spreading scheme (DDI_SPREAD_TILES / DDI_SPREAD_COLUMNS)
};
std::map<std::string, TuneResult> g_tune_cache;

}  // namespace

std::string tune_key_of(const Plan& p) {
  // kmax h_d only along the plan's own axes (a 2D plan's third axis is a placeholder)
  double kh[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < p.dim; ++a) kh[a] = p.desc.kmax * p.h[a];
  char buf[320];
  snprintf(buf, sizeof buf, "dev%d dim%d prec%d w%d n%d,%d,%d q%d,%d,%d kh%.12g,%.12g,%.12g chunk%d ell%d", p.device,
           p.dim, p.prec, p.w, p.n[0], p.n[1], p.n[2], p.desc.nr, p.desc.ntheta, p.desc.nphi, kh[0], kh[1], kh[2],
           p.desc.chunk, p.desc.ellipsoid);
  return buf;
}

namespace {

// candidate tiles (x, y, z) in fine cells; set_tile rounds each to a divisor of the fine
// grid that is at least w - 1, so duplicates after rounding are skipped
std::vector<std::array<int, 3>> tile_candidates(const Plan& p) {
  if (p.dim == 3) {
    if (p.prec == DDI_FP32)
      return {{32, 16, 16}, {32, 32, 8}, {16, 16, 16}, {64, 16, 8}, {64, 16, 16}, {32, 16, 8}, {32, 8, 16}, {16, 16, 32}};
    return {{16, 16, 16}, {32, 16, 16}, {16, 16, 32}, {32, 32, 16}};
  }
  return {{32, 16, 1}, {32, 32, 1}, {64, 16, 1}, {16, 16, 1}, {64, 32, 1}, {32, 8, 1}, {128, 16, 1}};
}

}  // namespace

// Column plans have fixed columns; the tuner picks the number of visits per work unit
// (more units balance the load better, fewer share fewer planes through partial slots).
int tune_column_chunk(Plan& p, cudaStream_t s) {
  const std::string key = tune_key_of(p) + " columns";
  std::unique_lock<std::mutex> lock(g_tune_mu);
  auto hit = g_tune_cache.find(key);
  if (hit != g_tune_cache.end()) {
    const TuneResult r = hit->second;
    lock.unlock();
    p.desc.chunk = r.chunk;
    DDI_TRY(build_spread_col(p, s));
    p.tuned_ms = r.ms;
    return DDI_OK;
  }
  int best = 0;
  double best_ms = 0.0;
  for (const int c : {32, 64, 128, 192, 256, 384, 512}) {
    p.desc.chunk = c;
    DDI_TRY(build_spread_col(p, s));
    float ms = 0.f;
    DDI_TRY(time_spread(p, s, 5, &ms));
    if (best == 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  g_tune_cache[key] = TuneResult{{{0, 0, 0}}, best, best_ms, DDI_SPREAD_COLUMNS};
  lock.unlock();
  p.desc.chunk = best;
  DDI_TRY(build_spread_col(p, s));
  p.tuned_ms = best_ms;
  return DDI_OK;
}

int tune_tiles(Plan& p, cudaStream_t s) {
  const std::string key = tune_key_of(p);
  std::unique_lock<std::mutex> lock(g_tune_mu);
  auto hit = g_tune_cache.find(key);
  if (hit != g_tune_cache.end()) {
    const TuneResult r = hit->second;
    lock.unlock();
    set_tile(p, r.tile.data());
    DDI_TRY(build_spread(p, s));
    p.tuned_ms = r.ms;
    return DDI_OK;
  }
  // tuning holds the lock: two tuners timing at once would disturb each other
  std::vector<std::array<int, 3>> tried;
  std::array<int, 3> best{{0, 0, 0}};
  double best_ms = 0.0;
  for (const auto& c : tile_candidates(p)) {
    set_tile(p, c.data());
    const std::array<int, 3> t{{p.tile[0], p.tile[1], p.tile[2]}};
    if (std::find(tried.begin(), tried.end(), t) != tried.end()) continue;
    tried.push_back(t);
    const int st = build_spread(p, s);
    if (st == DDI_ERR_ARG) continue;  // plane does not fit in shared memory
    DDI_TRY(st);
    float ms = 0.f;
    DDI_TRY(time_spread(p, s, 5, &ms));
    if (best[0] == 0 || ms < best_ms) {
      best = t;
      best_ms = ms;
    }
  }
  if (best[0] == 0) {
    set_error("spread-tile autotuner: no candidate tile fits in shared memory");
    return DDI_ERR_ARG;
  }
  g_tune_cache[key] = TuneResult{best, 0, best_ms, DDI_SPREAD_TILES};
  lock.unlock();
  set_tile(p, best.data());
  DDI_TRY(build_spread(p, s));
  p.tuned_ms = best_ms;
  return DDI_OK;
}

// 2D plans with the automatic scheme: the column spread at its best unit size against the
// tile spread at its best tile, the faster kept (the column spread wins on small fine
// grids, the tile spread on large ones; where the two cross depends on the node set)
int tune_scheme_2d(Plan& p, cudaStream_t s) {
  const std::string key = tune_key_of(p) + " scheme";
  {
    std::unique_lock<std::mutex> lock(g_tune_mu);
    auto hit = g_tune_cache.find(key);
    if (hit != g_tune_cache.end()) {
      const TuneResult r = hit->second;
      lock.unlock();
      drop_spread_lists(p);
      p.spread_kind = r.kind;
      if (r.kind == DDI_SPREAD_COLUMNS) {
        p.desc.chunk = r.chunk;
        DDI_TRY(build_spread_col(p, s));
      } else {
        set_tile(p, r.tile.data());
        DDI_TRY(build_spread(p, s));
      }
      p.tuned_ms = r.ms;
      return DDI_OK;
    }
  }
  const int user_chunk = p.desc.chunk;
  drop_spread_lists(p);
  p.spread_kind = DDI_SPREAD_COLUMNS;
  DDI_TRY(tune_column_chunk(p, s));
  const double col_ms = p.tuned_ms;
  const int col_chunk = p.desc.chunk;
  p.desc.chunk = user_chunk;
  drop_spread_lists(p);
  p.spread_kind = DDI_SPREAD_TILES;
  DDI_TRY(tune_tiles(p, s));
  TuneResult r{{{p.tile[0], p.tile[1], p.tile[2]}}, 0, p.tuned_ms, DDI_SPREAD_TILES};
  if (col_ms < p.tuned_ms) {
    drop_spread_lists(p);
    p.spread_kind = DDI_SPREAD_COLUMNS;
    p.desc.chunk = col_chunk;
    DDI_TRY(build_spread_col(p, s));
    p.tuned_ms = col_ms;
    r = TuneResult{{{0, 0, 0}}, col_chunk, col_ms, DDI_SPREAD_COLUMNS};
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = r;
  return DDI_OK;
}

int tune_spread_tile(Plan& p, cudaStream_t s) {
  if (p.dim == 2 && p.desc.spread == DDI_SPREAD_AUTO && columns_apply(p) && !p.batch_item)
    return tune_scheme_2d(p, s);
  if (p.spread_kind == DDI_SPREAD_COLUMNS) return tune_column_chunk(p, s);
  return tune_tiles(p, s);
}

}  // namespace ddi

using ddi::Plan;

struct ddi_batch_s {
  int device = 0;
  int flags = 0;
  std::vector<Plan*> plans;
  std::vector<std::vector<int>> branch;  // items of each side stream
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;            // the stream graphs are recorded on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> g_rho;        // pointers the executable graph was recorded with
  std::vector<void*> g_phi;
  long long records = 0, replays = 0;
};

namespace {

void free_batch(ddi_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (Plan* p : b->plans) {
    if (!p) continue;
    ddi::destroy_plan(*p);
    delete p;
  }
  for (cudaStream_t s : b->side)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

// relative cost of one DDI of a plan: the spread's (node, plane) pairs times w^2 taps,
// the interpolation's w^d taps per node and the fine-grid FFT passes
double item_cost(const Plan& p) {
  const double w = p.w;
  return (double)p.pairs * w * w + (double)p.Mh * std::pow(w, p.dim) + 40.0 * (double)p.fine_points();
}

template <typename T>
int run_item(Plan& p, const void* rho, void* phi, cudaStream_t s) {
  return ddi::run_ddi<T>(p, static_cast<const T*>(rho), static_cast<T*>(phi), s);
}

// fork from `origin`, every item on its side stream, join back into `origin`
int enqueue(ddi_batch_s* b, const void* const* rho, void* const* phi, cudaStream_t origin) {
  DDI_CUDA(cudaEventRecord(b->fork, origin));
  for (size_t k = 0; k < b->side.size(); ++k) {
    cudaStream_t s = b->side[k];
    DDI_CUDA(cudaStreamWaitEvent(s, b->fork, 0));
    for (int i : b->branch[k]) {
      Plan& p = *b->plans[i];
      DDI_TRY((p.prec == DDI_FP64 ? run_item<double>(p, rho[i], phi[i], s) : run_item<float>(p, rho[i], phi[i], s)));
    }
    DDI_CUDA(cudaEventRecord(b->join[k], s));
    DDI_CUDA(cudaStreamWaitEvent(origin, b->join[k], 0));
  }
  return DDI_OK;
}

int record_graph(ddi_batch_s* b, const void* const* rho, void* const* phi) {
  DDI_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  const int st = enqueue(b, rho, phi, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (st != DDI_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != DDI_OK) return st;
    ddi::set_error("cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
    return DDI_ERR_CUDA;
  }
  if (b->exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(b->exec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  if (!b->exec) {
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
    if (ei != cudaSuccess) {
      cudaGraphDestroy(g);
      b->exec = nullptr;
      ddi::set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(ei));
      return DDI_ERR_CUDA;
    }
  }
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph = g;
  const size_t n = b->plans.size();
  b->g_rho.assign(rho, rho + n);
  b->g_phi.assign(phi, phi + n);
  ++b->records;
  return DDI_OK;
}

int build_batch(ddi_batch_s* b, ddi_batch* out, const ddi_plan_desc* descs, int count, int flags, void* stream);
}  // namespace

extern "C" {

int ddi_batch_create(ddi_batch* out, const ddi_plan_desc* descs, int count, int flags, void* stream) {
  return ddi::guarded("ddi_batch_create", [&]() -> int {
    if (!out || !descs || count <= 0 || (flags & ~(DDI_BATCH_GRAPH | DDI_BATCH_AUTOTUNE)) != 0) {
      ddi::set_error("ddi_batch_create: out and descs must not be NULL, count > 0, flags a set of DDI_BATCH_*");
      return DDI_ERR_ARG;
    }
    *out = nullptr;
    ddi_batch_s* b = new (std::nothrow) ddi_batch_s();
    if (!b) {
      ddi::set_error("host allocation failed");
      return DDI_ERR_OOM;
    }
    b->flags = flags;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      ddi::set_error("ddi_batch_create: no current device");
      return DDI_ERR_CUDA;
    }
    try {
      return build_batch(b, out, descs, count, flags, stream);
    } catch (...) {
      free_batch(b);  // the plans and streams built before the failure
      throw;
    }
  });
}

}  // extern "C"

namespace {

// the body of ddi_batch_create once the batch object exists; failures free it (fail())
int build_batch(ddi_batch_s* b, ddi_batch* out, const ddi_plan_desc* descs, int count, int flags, void* stream) {
  b->plans.assign(count, nullptr);

  // plans are built by host threads (their tables and work lists are host work), each
  // with its own upload stream
  std::atomic<int> next{0};
  // the first failure of any thread, recorded without locks or allocation (nothing in the
  // threads may throw)
  std::atomic<int> first_status{DDI_OK};
  char first_msg[1024] = "";
  auto record = [&](int st, const char* msg) {
    int expect = DDI_OK;
    if (first_status.compare_exchange_strong(expect, st)) snprintf(first_msg, sizeof first_msg, "%s", msg);
  };
  auto worker = [&]() {
    cudaSetDevice(b->device);
    cudaStream_t s = nullptr;
    int st = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess ? DDI_OK : DDI_ERR_CUDA;
    if (st != DDI_OK) ddi::set_error("cudaStreamCreate failed");
    for (int i; st == DDI_OK && (i = next.fetch_add(1)) < count;) {
      Plan* p = new (std::nothrow) Plan();
      if (!p) {
        ddi::set_error("host allocation failed");
        st = DDI_ERR_OOM;
        break;
      }
      b->plans[i] = p;
      // an exception must not leave a worker thread
      st = ddi::guarded("ddi_batch_create", [&]() -> int { return ddi::create_plan(*p, &descs[i], s, false, true); });
      if (st != DDI_OK) ddi::set_error("batch item %d: %s", i, ddi::last_error());
    }
    if (st != DDI_OK) {
      record(st, ddi::last_error());
      next.store(count);
    }
    if (s) cudaStreamDestroy(s);
  };
  const int nthreads = std::max(1, std::min<int>(count, std::min(16u, std::max(1u, std::thread::hardware_concurrency()))));
  {
    // the shared counter balances any number of threads: if one cannot be started the
    // ones running (and this one) take its share
    std::vector<std::thread> pool;
    try {
      pool.reserve(nthreads);
      for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    } catch (...) {
    }
    worker();
    for (auto& t : pool) t.join();
  }
  auto fail = [&](int st) {
    free_batch(b);
    return st;
  };
  if (first_status.load() != DDI_OK) {
    ddi::set_error("%s", first_msg);
    return fail(first_status.load());
  }

  cudaStream_t s0 = static_cast<cudaStream_t>(stream);
  // autotune: one representative per shape is timed (one at a time on the GPU), the
  // other plans of that shape then rebuild their lists for the cached tile in parallel
  std::vector<int> tune_items;
  for (int i = 0; i < count; ++i)
    if ((flags & DDI_BATCH_AUTOTUNE) || descs[i].tile[0] < 0) tune_items.push_back(i);
  {
    std::map<std::string, int> firsts;
    for (int i : tune_items) firsts.emplace(ddi::tune_key_of(*b->plans[i]), i);
    for (auto& kv : firsts) {
      const int st = ddi::tune_spread_tile(*b->plans[kv.second], s0);
      if (st != DDI_OK) return fail(st);
    }
    std::atomic<int> nt{0};
    auto retune = [&]() {
      cudaSetDevice(b->device);
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        record(DDI_ERR_CUDA, "cudaStreamCreate failed");
        return;
      }
      for (int j; (j = nt.fetch_add(1)) < (int)tune_items.size();) {
        Plan& p = *b->plans[tune_items[j]];
        if (p.tuned_ms > 0.0) continue;
        const int st = ddi::guarded("ddi_batch_create", [&]() -> int { return ddi::tune_spread_tile(p, s); });
        if (st != DDI_OK) {
          record(st, ddi::last_error());
          nt.store((int)tune_items.size());
        }
      }
      cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    try {
      pool.reserve(nthreads);
      for (int t = 1; t < nthreads; ++t) pool.emplace_back(retune);
    } catch (...) {
    }
    retune();
    for (auto& t : pool) t.join();
    if (first_status.load() != DDI_OK) {
      ddi::set_error("%s", first_msg);
      return fail(first_status.load());
    }
  }
  // host copies only needed while building
  for (Plan* p : b->plans) {
    std::vector<ushort4>().swap(p->h_l0);
    std::vector<int>().swap(p->h_zcls);
    std::vector<int64_t>().swap(p->order);
    std::vector<double>().swap(p->quad.k);
    std::vector<double>().swap(p->quad.W);
  }

  // side streams: largest items first, each onto the least loaded stream
  const int nside = std::min(count, 8);
  b->side.assign(nside, nullptr);
  b->join.assign(nside, nullptr);
  b->branch.assign(nside, {});
  for (int k = 0; k < nside; ++k) {
    if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) != cudaSuccess) {
      ddi::set_error("ddi_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
      return fail(DDI_ERR_CUDA);
    }
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    ddi::set_error("ddi_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(DDI_ERR_CUDA);
  }
  std::vector<int> idx(count);
  for (int i = 0; i < count; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int x, int y) { return item_cost(*b->plans[x]) > item_cost(*b->plans[y]); });
  std::vector<double> load(nside, 0.0);
  for (int i : idx) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->branch[k].push_back(i);
    load[k] += item_cost(*b->plans[i]);
  }
  if (cudaStreamSynchronize(s0) != cudaSuccess) {
    ddi::set_error("ddi_batch_create: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(DDI_ERR_CUDA);
  }
  *out = b;
  return DDI_OK;
}

}  // namespace

extern "C" {

int ddi_batch_destroy(ddi_batch b) {
  if (b) {
    cudaDeviceSynchronize();
    free_batch(b);
  }
  return DDI_OK;
}

int ddi_batch_size(ddi_batch b) { return b ? (int)b->plans.size() : 0; }

int ddi_batch_get_info(ddi_batch b, int item, ddi_plan_info* info) {
  if (!b || !info || item < 0 || item >= (int)b->plans.size()) {
    ddi::set_error("ddi_batch_get_info: batch and info must not be NULL, 0 <= item < size");
    return DDI_ERR_ARG;
  }
  ddi::fill_info(*b->plans[item], info);
  return DDI_OK;
}

int ddi_batch_apply(ddi_batch b, const void* const* rho, void* const* phi, void* stream) {
  return ddi::guarded("ddi_batch_apply", [&]() -> int {
    if (!b || !rho || !phi) {
      ddi::set_error("ddi_batch_apply: batch, rho and phi must not be NULL");
      return DDI_ERR_ARG;
    }
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i)
      if (!rho[i] || !phi[i]) {
        ddi::set_error("ddi_batch_apply: rho[%zu] and phi[%zu] must be device pointers", i, i);
        return DDI_ERR_ARG;
      }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!(b->flags & DDI_BATCH_GRAPH)) return enqueue(b, rho, phi, s);
    const bool same = b->exec && std::equal(rho, rho + n, b->g_rho.begin()) && std::equal(phi, phi + n, b->g_phi.begin());
    if (!same) DDI_TRY(record_graph(b, rho, phi));
    DDI_CUDA(cudaGraphLaunch(b->exec, s));
    ++b->replays;
    return DDI_OK;
  });
}

int ddi_batch_graph_stats(ddi_batch b, long long* records, long long* launches) {
  if (!b) {
    ddi::set_error("ddi_batch_graph_stats: batch must not be NULL");
    return DDI_ERR_ARG;
  }
  if (records) *records = b->records;
  if (launches) *launches = b->replays;
  return DDI_OK;
}

}  // extern "C"

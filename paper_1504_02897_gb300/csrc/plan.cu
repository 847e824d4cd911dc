// Plan construction and the DDI entry points of the C ABI.
//
// A plan holds everything that depends only on the grid, the box, the dipole axes and
// the quadrature (Sec. 2.1, Eq. DDI-Trun1): the node tables (tables.cpp), for each node
// of one half of the antipodally closed set its first fine-grid tap, its kernel values
// psi_d at the w taps of each axis (FP64, rounded once) and its scale 2 h^d W_q, the
// deconvolution factors, the spread work list (per fine-grid tile, the nodes whose taps
// reach it, in order of their start relative to the tile, and the work units: one per
// tile plane, long ones cut into pieces that write partial planes), and all
// device workspace.  ddi_plan_create is the only call that allocates.
#include <algorithm>
#include <array>
#include <climits>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <numeric>

#include "common.cuh"

namespace ddi {

// ---- error reporting -----------------------------------------------------------------
// a fixed per-thread buffer: recording an error allocates nothing, so it is safe where
// memory has run out
namespace {
thread_local char g_err[1024] = "";
}
void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

namespace {

int dev_alloc(Plan& p, void** ptr, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes for %s failed", bytes, what);
    return DDI_ERR_OOM;
  }
  p.bytes += bytes;
  return DDI_OK;
}

template <typename V>
int upload(Plan& p, void** dst, const std::vector<V>& v, const char* what, cudaStream_t s) {
  DDI_TRY(dev_alloc(p, dst, sizeof(V) * std::max<size_t>(1, v.size()), what));
  if (!v.empty()) DDI_CUDA(cudaMemcpyAsync(*dst, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice, s));
  return DDI_OK;
}

// doubles -> the plan's real type
int upload_real(Plan& p, void** dst, const std::vector<double>& v, const char* what, cudaStream_t s,
                std::vector<float>* keep) {
  if (p.prec == DDI_FP64) return upload(p, dst, v, what, s);
  keep->assign(v.begin(), v.end());
  return upload(p, dst, *keep, what, s);
}

void choose_tile(Plan& p) {
  // Tiles are at least w - 1 cells per axis (a footprint reaches its own tile and the
  // next one only) and divide the fine grid.  3D: one warp per z-plane of the tile.
  auto pick = [](int want, int need, int nf) {
    for (int t = std::min(want, nf); t >= need && t >= 1; --t)
      if (nf % t == 0) return t;
    for (int t = need; t <= nf; ++t)
      if (nf % t == 0) return t;
    return nf;
  };
  const int need = p.w - 1;
  int want[3];
  if (p.dim == 3) {
    if (p.prec == DDI_FP32) {
      want[0] = 32; want[1] = 16; want[2] = 16;
    } else {
      want[0] = 16; want[1] = 16; want[2] = 16;
    }
  } else {
    want[0] = 32; want[1] = 16; want[2] = 1;
  }
  for (int d = 0; d < 3; ++d) {
    if (p.desc.tile[d] > 0) want[d] = p.desc.tile[d];
    if (d < p.dim && want[d] < need) want[d] = need;
    p.tile[d] = d < p.dim ? pick(want[d], need, p.nf[d]) : 1;
    p.ntile[d] = p.nf[d] / p.tile[d];
  }
  p.npl = p.dim == 3 ? p.tile[2] : 1;
}

void free_plan(Plan& p) {
  void* ptrs[] = {p.d_dirw,   p.d_l0,     p.d_psi,   p.d_scale, p.d_c,    p.d_deconv, p.d_ones,  p.d_fine,
                  p.d_deconv_x2, p.d_ones_x2,
                  p.d_partial,
                  p.d_visits, p.d_units, p.d_split, p.d_counter, p.d_psi1, p.d_rho, p.d_phi, p.d_work,
                  p.d_work2,  p.d_kin,   p.d_red,   p.d_io_in, p.d_io_out, p.d_cvis, p.d_cunits, p.d_cred,
                  p.d_cslots, p.d_cpart, p.d_nonfinite};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int i = 0; i < 8; ++i)
    if (p.d_tw[i]) {
      cudaFree(p.d_tw[i]);
      p.d_tw[i] = nullptr;
    }
  if (p.h_red) cudaFreeHost(p.h_red);
  if (p.ev_created)
    for (cudaEvent_t& e : p.mark_ev) cudaEventDestroy(e);
}

}  // namespace

void set_tile(Plan& p, const int want[3]) {
  for (int d = 0; d < 3; ++d) p.desc.tile[d] = want[d];
  choose_tile(p);
}

// Spread work lists for the plan's current tile: per tile the visit list, the work units
// (tile, owned plane) and the split units with their partial planes, uploaded to the
// device, and the spread's launch geometry.  Replaces the lists of an earlier tile (the
// spread-tile autotuner rebuilds them per candidate).
int build_spread(Plan& p, cudaStream_t stream) {
  const ddi_plan_desc& d = p.desc;
  const int dim = p.dim, W = p.w;
  const size_t rs = p.real_size(), cs = p.cx_size();
  const size_t warp_bytes = spread_warp_bytes(p.spread_plane_cells() * cs, spread_stage_bytes(W, rs));
  if (warp_bytes * (kSpreadThreads / 32) > 200 * 1024) {
    set_error("spread plane needs %zu bytes of shared memory per warp; choose a smaller tile", warp_bytes);
    return DDI_ERR_ARG;
  }
  // the previous lists may still be read by queued work on this stream
  DDI_CUDA(cudaStreamSynchronize(stream));
  for (void** q : {(void**)&p.d_visits, (void**)&p.d_units, (void**)&p.d_split, &p.d_partial})
    if (*q) {
      cudaFree(*q);
      *q = nullptr;
    }
  p.bytes -= p.spread_bytes;
  const size_t before = p.bytes;

  // spread visit lists: per tile, the nodes whose taps reach it with their starts relative
  // to the tile, ordered by (oz, oy, ox) so that each z-plane's nodes are one contiguous
  // range (3D)
  const int ntiles = p.ntile[0] * p.ntile[1] * p.ntile[2];
  std::vector<std::vector<std::pair<int64_t, int4>>> lists(ntiles);
  for (int64_t i = 0; i < p.Mh; ++i) {
    const int lv[3] = {p.h_l0[i].x, p.h_l0[i].y, p.h_l0[i].z};
    int ta[3][2], nt[3];
    for (int a = 0; a < 3; ++a) {
      const int l = a < dim ? lv[a] : 0;
      const int w = a < dim ? W : 1;
      const int sh = p.ntile[a] > 1 ? p.tile[a] / 2 : 0;  // lattice shift of tile_origin
      ta[a][0] = ((l + sh) % p.nf[a]) / p.tile[a];
      ta[a][1] = ((l + w - 1 + sh) % p.nf[a]) / p.tile[a];
      nt[a] = ta[a][1] != ta[a][0] ? 2 : 1;
    }
    for (int cz = 0; cz < nt[2]; ++cz)
      for (int cy = 0; cy < nt[1]; ++cy)
        for (int cx = 0; cx < nt[0]; ++cx) {
          const int bx = ta[0][cx], by = ta[1][cy], bz = ta[2][cz];
          const int t = (bz * p.ntile[1] + by) * p.ntile[0] + bx;
          const int ox = rel_start(lv[0], tile_origin(bx, p.tile[0], p.ntile[0], p.nf[0]), p.nf[0], W);
          const int oy = rel_start(lv[1], tile_origin(by, p.tile[1], p.ntile[1], p.nf[1]), p.nf[1], W);
          const int oz = dim == 3 ? rel_start(lv[2], tile_origin(bz, p.tile[2], p.ntile[2], p.nf[2]), p.nf[2], W) : 0;
          // starts lie in [-15, 2048): offset by 32 into 12-bit fields
          const int64_t key = dim == 3 ? (((int64_t)oz + 32) * 4096 + (oy + 32)) * 4096 + (ox + 32)
                                       : ((int64_t)oy + 32) * 4096 + (ox + 32);
          lists[t].push_back(std::make_pair(key, make_int4((int)i, ox, oy, oz)));
        }
  }
  long long total = 0;
  for (auto& L : lists) {
    std::stable_sort(L.begin(), L.end(), [](const std::pair<int64_t, int4>& a, const std::pair<int64_t, int4>& b) {
      return a.first < b.first;
    });
    total += (long long)L.size();
  }
  p.visits = total;
  if (total > (long long)INT32_MAX - 1) {
    // visit ranges are 32-bit on the device
    set_error("%lld spread visits exceed the 32-bit visit lists; use fewer quadrature nodes", total);
    return DDI_ERR_ARG;
  }
  // 2D: one unit per tile (the whole tile is the plane); 3D: one per z-plane
  const bool wrap_owned = dim == 3 ? p.ntile[2] == 1 : true;
  std::vector<int4> visits;
  visits.reserve(total);
  // work units (tile, owned plane): the list entries whose taps along the owned axis cover
  // the plane form one contiguous range (lists are sorted by the owned start)
  std::vector<SpreadUnit> units;
  long long pairs = 0;
  for (int t = 0; t < ntiles; ++t) {
    const int beg = (int)visits.size();
    for (auto& e : lists[t]) visits.push_back(e.second);
    const int end = (int)visits.size();
    auto owned = [&](int k) { return visits[k].w; };
    for (int pl = 0; pl < p.npl; ++pl) {
      int lo = beg, hi = end;
      if (!wrap_owned) {
        int l = beg, h = end;
        while (l < h) {
          const int m = (l + h) / 2;
          if (owned(m) < pl - W + 1) l = m + 1; else h = m;
        }
        lo = l;
        h = end;
        while (l < h) {
          const int m = (l + h) / 2;
          if (owned(m) <= pl) l = m + 1; else h = m;
        }
        hi = l;
      }
      units.push_back(SpreadUnit{t, pl, lo, hi, -1});
      pairs += hi - lo;
    }
  }
  p.pairs = pairs;
  // long units are cut into pieces that write partial planes (summed by k_reduce)
  // (at least 1024 visits in 3D, 256 in 2D: a hot 2D tile's pieces run one after another
  // on one warp each, so shorter pieces shorten the launch's critical path)
  p.chunk = d.chunk > 0 ? d.chunk : (int)std::max<long long>(dim == 2 ? 256 : 1024, pairs / (152LL * 32 * 2));
  std::vector<SpreadUnit> work;
  std::vector<SplitUnit> split;
  int slot = 0;
  for (const SpreadUnit& U : units) {
    const int v = U.hi - U.lo;
    if (v <= p.chunk) {
      work.push_back(U);
    } else {
      const int nch = (v + p.chunk - 1) / p.chunk;
      split.push_back(SplitUnit{U.tile, U.plane, slot, nch});
      for (int c = 0; c < nch; ++c)
        work.push_back(SpreadUnit{U.tile, U.plane, U.lo + c * p.chunk, std::min(U.hi, U.lo + (c + 1) * p.chunk), slot + c});
      slot += nch;
    }
  }
  // largest units first: the persistent spread takes them in this order
  std::stable_sort(work.begin(), work.end(),
                   [](const SpreadUnit& a, const SpreadUnit& b) { return (a.hi - a.lo) > (b.hi - b.lo); });
  p.nunits = (int)work.size();
  p.nsplit = (int)split.size();
  p.nslots = slot;

  DDI_TRY(upload(p, (void**)&p.d_visits, visits, "visit lists", stream));
  DDI_TRY(upload(p, (void**)&p.d_units, work, "work units", stream));
  DDI_TRY(upload(p, (void**)&p.d_split, split, "split units", stream));
  const size_t plane_cells = (size_t)p.tile[0] * p.tile[1];
  DDI_TRY(dev_alloc(p, &p.d_partial, cs * plane_cells * std::max(1, p.nslots), "partial planes"));
  p.spread_bytes = p.bytes - before;
  // the host vectors above die with this frame
  DDI_CUDA(cudaStreamSynchronize(stream));
  return configure_kernels(p);
}

// Whether the column spread applies: FP32 plans whose fine grid holds whole columns and is
// wide enough that a footprint meets a column (or a window) in one contiguous piece.  2D
// columns carry no compensated variant (compensated 2D plans use the tile spread).
bool columns_apply(const Plan& p) {
  if (p.prec != DDI_FP32 || p.w > 16 || p.nf[0] % kColX != 0 || p.nf[0] < kColX + p.w - 1) return false;
  if (p.dim == 2) return p.nf[1] >= p.w && p.desc.compensated == 0;
  return p.dim == 3 && p.nf[1] % kColY == 0 && p.nf[1] >= kColY + p.w - 1 && p.nf[2] >= p.w;
}

// Frees the spread lists of both schemes (the autotuner switches a 2D plan between them).
void drop_spread_lists(Plan& p) {
  for (void** q : {(void**)&p.d_visits, (void**)&p.d_units, (void**)&p.d_split, &p.d_partial, (void**)&p.d_cvis,
                   (void**)&p.d_cunits, (void**)&p.d_cred, (void**)&p.d_cslots, &p.d_cpart})
    if (*q) {
      cudaFree(*q);
      *q = nullptr;
    }
  p.bytes -= p.spread_bytes;
  p.spread_bytes = 0;
}

// Column spread lists.  3D: columns of kColX x kColY cells in x-y run the whole z axis (the
// window axis); 2D: columns of kColX cells in x run the whole y axis.  Every processed node
// visits the columns its cross-axis taps reach; a column's visits are sorted by the node's
// first tap along the window axis, then (3D) by z class, then by node.  The visits are cut
// into units of at most `chunk` visits; unit c writes the planes (2D: rows) [a_c, e_c), a_c =
// its first visit's first tap, e_c the end of its last footprint extended over the gap to the
// next unit (at most 64 planes ahead; longer gaps and empty columns get units without visits
// that only write zeros).  A plane that several units touch (their footprints overlap at unit
// boundaries, and the last unit of a column wraps onto the first) is a leading or trailing
// plane of each of them: those go to partial slots and a reduce entry sums them in unit order;
// every other plane is written by its one unit.  Every fine cell is written once per apply.
int build_spread_col(Plan& p, cudaStream_t stream) {
  const bool d3 = p.dim == 3;
  const int W = p.w, nfx = p.nf[0], nfy = p.nf[1];
  const int nfz = p.nf[p.dim - 1];  // the window axis: z (3D), y (2D)
  const int cy_cells = d3 ? kColY : 1;
  const int ncx = nfx / kColX, ncy = d3 ? nfy / kColY : 1, ncol = ncx * ncy;
  DDI_CUDA(cudaStreamSynchronize(stream));
  for (void** q : {(void**)&p.d_cvis, (void**)&p.d_cunits, (void**)&p.d_cred, (void**)&p.d_cslots, &p.d_cpart})
    if (*q) {
      cudaFree(*q);
      *q = nullptr;
    }
  p.bytes -= p.spread_bytes;
  const size_t before = p.bytes;
  // visits: key (column, first window-axis tap) and the packed entry
  auto span = [&](int l, int nf, int B, int* first) {  // blocks of B cells a footprint from l reaches
    *first = l / B;
    const int last = ((l + W - 1) % nf) / B;
    int k = last - *first;
    if (k < 0) k += nf / B;
    return k + 1;
  };
  auto yspan = [&](int l, int* first) {  // 2D: the one column row
    if (d3) return span(l, nfy, kColY, first);
    *first = 0;
    return 1;
  };
  auto wtap = [&](const ushort4& l) { return d3 ? (int)l.z : (int)l.y; };
  std::vector<int> count(ncol + 1, 0);
  for (int64_t i = 0; i < p.Mh; ++i) {
    int fx, fy;
    const int kx = span(p.h_l0[i].x, nfx, kColX, &fx), ky = yspan(p.h_l0[i].y, &fy);
    for (int b = 0; b < ky; ++b)
      for (int a = 0; a < kx; ++a) ++count[((fy + b) % ncy) * ncx + (fx + a) % ncx];
  }
  std::vector<int> start(ncol + 1, 0);
  for (int c = 0; c < ncol; ++c) start[c + 1] = start[c] + count[c];
  const long long total = start[ncol];
  if (total > (long long)INT32_MAX - 1 || p.Mh > (int64_t)INT32_MAX) {
    set_error("%lld column-spread visits exceed the 32-bit visit lists; use fewer quadrature nodes", total);
    return DDI_ERR_ARG;
  }
  std::vector<int2> vis((size_t)total);
  {
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < p.Mh; ++i) {
      const ushort4 l = p.h_l0[i];
      int fx, fy;
      const int kx = span(l.x, nfx, kColX, &fx), ky = yspan(l.y, &fy);
      for (int b = 0; b < ky; ++b)
        for (int a = 0; a < kx; ++a) {
          const int bx = (fx + a) % ncx, by = (fy + b) % ncy;
          const int ox = rel_start(l.x, bx * kColX, nfx, W), oy = d3 ? rel_start(l.y, by * kColY, nfy, W) : 0;
          if (ox < -(W - 1) || ox >= kColX || oy < -(W - 1) || oy >= cy_cells) {
            set_error("column spread: footprint offset (%d, %d) outside its column", ox, oy);
            return DDI_ERR_INTERNAL;
          }
          vis[fill[by * ncx + bx]++] = make_int2((int)i, (wtap(l) << 13) | ((oy + 16) << 6) | (ox + 16));
        }
    }
  }
  // per column: by first window-axis tap, then z class (3D: nodes with the same first tap and
  // bit-identical psi_z rows, e.g. one quadrature ring; 2D: one class), then node (the visits
  // are in node order already); bit 12 marks the first visit of each run of one (tap, class)
  for (int c = 0; c < ncol; ++c) {
    auto b = vis.begin() + start[c], e = vis.begin() + start[c + 1];
    std::stable_sort(b, e, [&](const int2& u, const int2& v) {
      const int su = u.y >> 13, sv = v.y >> 13;
      return su != sv ? su < sv : p.h_zcls[u.x] < p.h_zcls[v.x];
    });
    for (auto it = b; it != e; ++it)
      if (it == b || (it->y >> 13) != ((it - 1)->y >> 13) || p.h_zcls[it->x] != p.h_zcls[(it - 1)->x])
        it->y |= 1 << 12;
  }
  const int cap = p.desc.chunk > 0 ? p.desc.chunk : 256;
  const int lmax = std::min(64, nfz);
  std::vector<ColUnit> units;
  std::vector<ColRed> red;
  std::vector<int> slots;  // per unit-local shared plane: its partial slot
  int nslot = 0, nslot_e = 0;
  std::vector<int> tc(nfz);
  std::vector<std::vector<int>> contrib(nfz);
  for (int c = 0; c < ncol; ++c) {
    const int b0 = start[c], b1 = start[c + 1];
    const size_t u0 = units.size();
    if (b0 == b1) {
      // an empty column is written as zeros, unless none of its x or y lines holds a tap (the
      // NUFFT's passes neither transform nor read those lines)
      bool in_y = !d3, in_x = false;  // a 2D column holds every y line
      for (int r = 0; d3 && r < kColY; ++r) {
        int d = (c / ncx) * kColY + r - p.yr[0];
        if (d < 0) d += nfy;
        in_y = in_y || d < p.yr[1];
      }
      for (int r = 0; r < kColX; ++r) {
        int d = (c % ncx) * kColX + r - p.xr[0];
        if (d < 0) d += nfx;
        in_x = in_x || d < p.xr[1];
      }
      const bool needed = in_x && in_y;
      if (needed)
        for (int z = 0; z < nfz; z += lmax) units.push_back(ColUnit{c, b0, b0, z, std::min(nfz, z + lmax), 0, 0, 0});
      continue;
    }
    // visit chunks and their planes [a, b) (b = last first tap + w)
    std::vector<std::array<int, 4>> ch;  // lo, hi, a, b
    for (int k = b0; k < b1; k += cap) {
      const int hi = std::min(b1, k + cap);
      ch.push_back({{k, hi, vis[k].y >> 13, (vis[hi - 1].y >> 13) + W}});
    }
    const int nch = (int)ch.size();
    for (int k = 0; k < nch; ++k) {
      const int a = ch[k][2];
      const int next = k + 1 < nch ? ch[k + 1][2] : ch[0][2] + nfz;
      const int e = std::max(ch[k][3], std::min(next, a + lmax));
      units.push_back(ColUnit{c, ch[k][0], ch[k][1], a, e, 0, 0, 0});
      for (int z = e; z < next; z += lmax) units.push_back(ColUnit{c, ch[k][1], ch[k][1], z, std::min(next, z + lmax), 0, 0, 0});
    }
    // planes touched by several units
    std::fill(tc.begin(), tc.end(), 0);
    for (size_t u = u0; u < units.size(); ++u)
      for (int z = units[u].z0; z < units[u].z1; ++z) ++tc[z % nfz];
    for (size_t u = u0; u < units.size(); ++u) {
      ColUnit& U = units[u];
      const int len = U.z1 - U.z0;
      int lo = 0, hi = 0;
      while (lo < len && tc[(U.z0 + lo) % nfz] > 1) ++lo;
      if (lo < len)
        while (hi < len - lo && tc[(U.z1 - 1 - hi) % nfz] > 1) ++hi;
      for (int r = lo; r < len - hi; ++r)
        if (tc[(U.z0 + r) % nfz] != 1) {
          set_error("column spread: shared plane inside a unit's window");
          return DDI_ERR_INTERNAL;
        }
      U.plo = lo;
      U.phi = hi;
      U.slot0 = nslot;
      for (int r = 0; r < lo; ++r) contrib[(U.z0 + r) % nfz].push_back(nslot + r);
      for (int r = 0; r < hi; ++r) contrib[(U.z1 - hi + r) % nfz].push_back(nslot + lo + r);
      nslot += lo + hi;
      slots.resize(nslot);
    }
    // slots entry-major: the contributions to one plane are contiguous, in unit order;
    // slots[] maps each unit's k-th shared plane (unit-local numbering) to its slot
    for (int z = 0; z < nfz; ++z) {
      if (contrib[z].empty()) continue;
      red.push_back(ColRed{c, z, nslot_e, (int)contrib[z].size()});
      for (int q : contrib[z]) slots[q] = nslot_e++;
      contrib[z].clear();
    }
  }
  // costliest units first.  3D: visits plus the planes each writes.  2D: the four lane
  // groups share a run (one first y tap), so a run of L visits takes ceil(L / 4) steps; a
  // unit costs about 4 per step, 3 per run and 5 per row it writes (relative instruction
  // counts of the kernel's visit step, run start and row flush)
  {
    std::vector<long long> cost(units.size());
    for (size_t u = 0; u < units.size(); ++u) {
      const ColUnit& U = units[u];
      if (d3) {
        cost[u] = (long long)(U.hi - U.lo) + (U.z1 - U.z0);
        continue;
      }
      long long steps = 0, runs = 0;
      int len = 0;
      for (int k = U.lo; k < U.hi; ++k) {
        if (k > U.lo && ((vis[k].y >> 12) & 1)) {
          steps += (len + 3) / 4;
          ++runs;
          len = 0;
        }
        ++len;
      }
      if (len > 0) {
        steps += (len + 3) / 4;
        ++runs;
      }
      cost[u] = 4 * steps + 3 * runs + 5LL * (U.z1 - U.z0);
    }
    std::vector<size_t> ord(units.size());
    std::iota(ord.begin(), ord.end(), (size_t)0);
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<ColUnit> sorted(units.size());
    for (size_t k = 0; k < ord.size(); ++k) sorted[k] = units[ord[k]];
    units.swap(sorted);
  }
  if (units.size() > (size_t)INT32_MAX || slots.size() > (size_t)INT32_MAX) {
    set_error("column spread: work list too long");
    return DDI_ERR_ARG;
  }
  p.visits = total;
  p.pairs = total;
  p.chunk = cap;
  p.ncunits = (int)units.size();
  p.ncred = (int)red.size();
  p.ncslots = nslot;
  DDI_TRY(upload(p, (void**)&p.d_cvis, vis, "column visits", stream));
  DDI_TRY(upload(p, (void**)&p.d_cunits, units, "column units", stream));
  DDI_TRY(upload(p, (void**)&p.d_cred, red, "column reduce entries", stream));
  DDI_TRY(upload(p, (void**)&p.d_cslots, slots, "column slot lists", stream));
  DDI_TRY(dev_alloc(p, &p.d_cpart, p.cx_size() * kColX * cy_cells * (size_t)std::max(1, nslot),
                    "column partial planes"));
  p.spread_bytes = p.bytes - before;
  DDI_CUDA(cudaStreamSynchronize(stream));
  return configure_kernels(p);
}

int create_plan(Plan& p, const ddi_plan_desc* desc_in, cudaStream_t stream, bool gpe, bool batch_item) {
  std::string err;
  {
    const int st = normalise_desc(desc_in, &p.desc, &err);
    if (st != DDI_OK) {
      set_error("%s", err.c_str());
      return st;
    }
  }
  const ddi_plan_desc& d = p.desc;
  DDI_CUDA(cudaGetDevice(&p.device));
  p.dim = d.dim;
  p.prec = d.precision;
  p.dv = 1.0;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = a < d.dim ? d.n[a] : 1;
    p.nf[a] = a < d.dim ? 2 * d.n[a] : 1;
    p.h[a] = a < d.dim ? d.len[a] / (double)d.n[a] : 1.0;
    if (a < d.dim) p.dv *= p.h[a];
  }
  p.w = kernel_width(d);
  p.beta = kernel_beta(p.w);
  // every tap l of a ball node with |k_a| <= kmax lies within |l| <= kmax h nf / (2 pi) + w/2 (first
  // tap ceil(s - w/2), last tap + w - 1)
  split_band(d, p.w, p.band);
  build_quadrature(d, &p.quad, /*keep_dirs=*/gpe);
  p.M = p.quad.M;
  choose_tile(p);
  const int dim = d.dim, W = p.w;
  if (d.spread == DDI_SPREAD_COLUMNS && !columns_apply(p)) {
    set_error("the column spread needs an FP32 plan whose fine grid is a multiple of %d cells in x (3D: %d x %d in "
              "x-y) and at least w + %d cells along x (3D: w + %d along y and w along z; 2D: w along y), and no "
              "compensated arithmetic in 2D",
              kColX, kColX, kColY, kColX - 1, kColY - 1);
    return DDI_ERR_ARG;
  }
  // automatic choice: columns in 3D.  In 2D, a plan on its own takes columns only up to 512^2
  // fine cells; above that the tile spread measured faster alone (the 2D column's runs of one
  // first y tap are short there, so three of its four lane groups idle), and its autotuner
  // times both schemes.  Batch items take columns at every size: they run beside the other
  // items' kernels, and the 96-density batch measured 13.3 ms with columns against 15.5 ms
  // with tiles (the faster tiles alone) and 15.2 ms with the size rule
  p.batch_item = batch_item;
  p.spread_kind = columns_apply(p) && (d.spread == DDI_SPREAD_COLUMNS ||
                                       (d.spread == DDI_SPREAD_AUTO &&
                                        (p.dim == 3 || batch_item || (long long)p.nf[0] * p.nf[1] <= 512LL * 512)))
                      ? DDI_SPREAD_COLUMNS
                      : DDI_SPREAD_TILES;
  // compensated FP32 arithmetic: head + tail twiddles in the NUFFT's fine-grid passes and
  // compensated (Kahan) plane sums in the column spread
  p.precise_nufft = d.compensated != 0 && d.precision == DDI_FP32;
  p.col_comp = d.compensated != 0;

  // one node of each (k, -k) pair: the first half of the azimuth
  const int nphi = d.nphi, half = nphi / 2;
  std::vector<int64_t> qs;
  qs.reserve(p.M / 2);
  for (int64_t q = 0; q < p.M; ++q)
    if ((q % nphi) < half) qs.push_back(q);
  p.Mh = (int64_t)qs.size();

  // first taps (wrapped), kernel values and scales; processing order groups nodes by
  // their first-tap tile (spatial locality of the interpolation reads)
  std::vector<int> l0w(3 * p.Mh, 0);
  std::vector<double> fr(3 * p.Mh, 0.0);
  std::vector<int64_t> okey(p.Mh);
  for (int64_t i = 0; i < p.Mh; ++i) {
    const int64_t q = qs[i];
    for (int a = 0; a < dim; ++a) {
      const double k = p.quad.k[dim * q + a];
      const int64_t l0 = fine_start(k, p.h[a], p.nf[a], W);
      const double s = k * ((p.h[a] * (double)p.nf[a]) / (2.0 * M_PI));
      fr[3 * i + a] = s - (double)l0;  // tap a sits at x = l0 + a - s
      l0w[3 * i + a] = (int)(((l0 % p.nf[a]) + p.nf[a]) % p.nf[a]);
    }
    const int bx = l0w[3 * i] / p.tile[0], by = l0w[3 * i + 1] / p.tile[1], bz = l0w[3 * i + 2] / p.tile[2];
    const int64_t bin = ((int64_t)bz * p.ntile[1] + by) * p.ntile[0] + bx;
    const int64_t key = ((int64_t)l0w[3 * i + 2] * p.nf[1] + l0w[3 * i + 1]) * p.nf[0] + l0w[3 * i];
    okey[i] = bin * p.fine_points() + key;
  }
  std::vector<int64_t> perm(p.Mh);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return okey[a] < okey[b]; });

  p.order.resize(p.Mh);
  std::vector<ushort4>& l0s = p.h_l0;
  l0s.assign(p.Mh, ushort4{});
  std::vector<double> psi((size_t)p.Mh * 3 * W, 1.0), scale(p.Mh);
  const double hw = 0.5 * (double)W;
  // z classes: nodes whose first z tap and fractional z offset are equal have the same psi_z
  // row (computed by the same operations), so the column spread can sum them before psi_z
  p.h_zcls.assign(p.Mh, 0);
  {
    std::vector<std::pair<std::pair<int, uint64_t>, int64_t>> zk((size_t)p.Mh);
    for (int64_t i = 0; i < p.Mh; ++i) {
      uint64_t bits = 0;
      const double f = dim == 3 ? fr[3 * perm[i] + 2] : 0.0;
      std::memcpy(&bits, &f, sizeof bits);
      zk[i] = std::make_pair(std::make_pair(dim == 3 ? l0w[3 * perm[i] + 2] : 0, bits), i);
    }
    std::sort(zk.begin(), zk.end());
    int cls = -1;
    for (size_t k = 0; k < zk.size(); ++k) {
      if (k == 0 || zk[k].first != zk[k - 1].first) ++cls;
      p.h_zcls[zk[k].second] = cls;
    }
  }
  for (int64_t i = 0; i < p.Mh; ++i) {
    const int64_t o = perm[i];
    p.order[i] = qs[o];
    l0s[i] = make_ushort4((unsigned short)l0w[3 * o], (unsigned short)l0w[3 * o + 1],
                          (unsigned short)l0w[3 * o + 2], 0);
    for (int a = 0; a < 3; ++a)
      for (int t = 0; t < W; ++t) {
        double v = a < dim ? 0.0 : (t == 0 ? 1.0 : 0.0);
        if (a < dim) {
          const double z = ((double)t - fr[3 * o + a]) / hw;
          if (z * z < 1.0) v = std::exp(p.beta * (std::sqrt((1.0 - z) * (1.0 + z)) - 1.0));
        }
        psi[((size_t)i * 3 + a) * W + t] = v;
      }
    scale[i] = 2.0 * p.dv * p.quad.W[qs[o]];
  }

  // the shortest cyclic range of fine y lines holding every tap (the complement of the
  // longest run of lines no tap reaches); every line for split plans, whose smooth part
  // shares the passes' geometry with full transforms
  {
    const int nfy = p.nf[1];
    std::vector<char> hit(nfy, 0);
    for (int64_t i = 0; i < p.Mh; ++i)
      for (int t = 0; t < (dim >= 2 ? W : 1); ++t) hit[(l0s[i].y + t) % nfy] = 1;
    int best = 0, best_end = 0;  // longest cyclic run of untouched lines, ending before best_end
    int run = 0;
    for (int k = 0; k < 2 * nfy; ++k) {
      run = hit[k % nfy] ? 0 : std::min(run + 1, nfy);
      if (run > best) {
        best = run;
        best_end = (k + 1) % nfy;
      }
    }
    if (p.split() || best == 0 || p.Mh == 0) {
      p.yr[0] = 0;
      p.yr[1] = nfy;
    } else {
      p.yr[0] = best_end;  // the first touched line after the gap
      p.yr[1] = nfy - best;
    }
    p.xr[0] = 0;
    p.xr[1] = p.nf[0];
    // split plans with a band: the ball's taps lie within |l| <= band of k = 0 along x and y
    if (p.split() && p.dim == 3 && p.band[0] > 0 && p.band[1] > 0) {
      p.xr[0] = p.nf[0] - p.band[0];
      p.xr[1] = 2 * p.band[0] + 1;
      p.yr[0] = nfy - p.band[1];
      p.yr[1] = 2 * p.band[1] + 1;
    }
  }

  // deconvolution factors 1/psihat(2 pi j'/nf), j' = j - n/2
  std::vector<double> dc;
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < p.n[a]; ++j)
      dc.push_back(p.n[a] == 1 ? 1.0
                               : 1.0 / es_kernel_hat(2.0 * M_PI * (double)(j - p.n[a] / 2) / (double)p.nf[a], W, p.beta));

  // device memory
  const size_t rs = p.real_size(), cs = p.cx_size();
  std::vector<float> k1, k2;
  DDI_TRY(upload(p, &p.d_l0, l0s, "node taps", stream));
  DDI_TRY(upload_real(p, &p.d_psi, psi, "kernel values", stream, &k1));
  DDI_TRY(upload_real(p, &p.d_scale, scale, "node scales", stream, &k2));
  std::vector<NodeDir> dirw;
  if (gpe) {
    // per processed node, what its weight is rebuilt from for other axes
    dirw.resize(p.Mh);
    for (int64_t i = 0; i < p.Mh; ++i) {
      const double* o = &p.quad.dirw[4 * p.order[i]];
      dirw[i] = NodeDir{o[0], o[1], o[2], o[3]};
    }
    DDI_TRY(upload(p, (void**)&p.d_dirw, dirw, "node directions", stream));
  }
  // deconvolution factors stay FP64 in both precisions; FP32 plans also get the x factors
  // as FP32 head + tail pairs (applied so that only the final product is rounded)
  auto pairs = [](const std::vector<double>& v, int n) {
    std::vector<float2> out((size_t)n);
    for (int j = 0; j < n; ++j) {
      const float hi = (float)v[j];
      out[j] = make_float2(hi, (float)(v[j] - (double)hi));
    }
    return out;
  };
  DDI_TRY(upload(p, &p.d_deconv, dc, "deconvolution", stream));
  std::vector<float2> dcx2 = pairs(dc, p.n[0]);
  DDI_TRY(upload(p, &p.d_deconv_x2, dcx2, "deconvolution pairs", stream));
  std::vector<double> ones;
  std::vector<float2> ones2;
  if (p.split()) {
    ones.assign((size_t)p.n[0] + p.n[1] + p.n[2], 1.0);
    ones2 = pairs(ones, p.n[0]);
    DDI_TRY(upload(p, &p.d_ones, ones, "unit factors", stream));
    DDI_TRY(upload(p, &p.d_ones_x2, ones2, "unit factor pairs", stream));
  }
  DDI_TRY(dev_alloc(p, (void**)&p.d_counter, sizeof(int), "unit counter"));
  DDI_TRY(dev_alloc(p, (void**)&p.d_nonfinite, sizeof(int), "non-finite record"));
  DDI_CUDA(cudaMemsetAsync(p.d_nonfinite, 0, sizeof(int), stream));
  DDI_TRY(dev_alloc(p, &p.d_c, cs * p.Mh, "node values"));
  DDI_TRY(dev_alloc(p, &p.d_fine, cs * p.fine_points(), "fine grid"));
  for (int a = 0; a < 3; ++a) {
    if (p.nf[a] > 1) DDI_TRY(make_twiddles(p, p.nf[a]));
    if (p.n[a] > 1) DDI_TRY(make_twiddles(p, p.n[a]));
  }
  // the host vectors above die with this frame: finish the uploads first
  DDI_CUDA(cudaStreamSynchronize(stream));
  std::vector<double>().swap(p.quad.dirw);
  DDI_TRY(p.spread_kind == DDI_SPREAD_COLUMNS ? build_spread_col(p, stream) : build_spread(p, stream));
  if (!gpe) return DDI_OK;
  const size_t N = (size_t)p.grid_points();
  DDI_TRY(dev_alloc(p, &p.d_psi1, cs * N, "gpe psi1"));
  DDI_TRY(dev_alloc(p, &p.d_rho, rs * N, "gpe rho"));
  DDI_TRY(dev_alloc(p, &p.d_phi, rs * N, "gpe phi"));
  DDI_TRY(dev_alloc(p, &p.d_work, cs * N, "gpe work"));
  DDI_TRY(dev_alloc(p, &p.d_work2, cs * N, "gpe work2"));
  DDI_TRY(dev_alloc(p, &p.d_kin, cs * (p.n[0] + p.n[1] + p.n[2]), "kinetic tables"));
  p.red_blocks = 1024;
  DDI_TRY(dev_alloc(p, (void**)&p.d_red, sizeof(double) * 16 * (p.red_blocks + 1), "reductions"));
  if (cudaMallocHost((void**)&p.h_red, sizeof(double) * 64) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocHost failed");
    return DDI_ERR_OOM;
  }
  DDI_TRY(dev_alloc(p, &p.d_io_in, rs * N, "host io in"));
  DDI_TRY(dev_alloc(p, &p.d_io_out, rs * N, "host io out"));
  p.gpe_ready = true;
  return DDI_OK;
}

namespace {

// Node scales 2 h^d W_q for the axes (n, m): the symbol and W in the order of operations
// of build_quadrature (explicitly rounded FP64 operations, no contraction), so the result
// is bit-identical to a plan built with these axes.
template <typename T>
__global__ void k_set_axes(const NodeDir* __restrict__ dirw, T* __restrict__ scale, long long count, int dim,
                           double n0, double n1, double n2, double m0, double m1, double m2, double nm,
                           double divisor, double two_dv) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const NodeDir o = dirw[i];
  double sym;
  if (dim == 3) {
    const double nk = __dadd_rn(__dadd_rn(__dmul_rn(n0, o.x), __dmul_rn(n1, o.y)), __dmul_rn(n2, o.z));
    const double mk = __dadd_rn(__dadd_rn(__dmul_rn(m0, o.x), __dmul_rn(m1, o.y)), __dmul_rn(m2, o.z));
    sym = __dsub_rn(__dmul_rn(3.0, __dmul_rn(nk, mk)), nm);
  } else {
    const double nk = __dadd_rn(__dmul_rn(n0, o.x), __dmul_rn(n1, o.y));
    const double mk = __dadd_rn(__dmul_rn(m0, o.x), __dmul_rn(m1, o.y));
    sym = __dmul_rn(1.5, __dsub_rn(__dmul_rn(nk, mk), __dmul_rn(n2, m2)));
  }
  const double W = __ddiv_rn(__dmul_rn(o.w, sym), divisor);
  scale[i] = (T)__dmul_rn(two_dv, W);
}

}  // namespace

int set_axes(Plan& p, const double* axis_n, const double* axis_m, cudaStream_t s) {
  if (!p.d_dirw) {
    set_error("ddi_plan_set_axes: this plan keeps no node directions");
    return DDI_ERR_ARG;
  }
  ddi_plan_desc d = p.desc;
  for (int a = 0; a < 3; ++a) {
    d.axis_n[a] = axis_n[a];
    d.axis_m[a] = axis_m ? axis_m[a] : 0.0;
  }
  ddi_plan_desc nd;
  std::string err;
  const int st = normalise_desc(&d, &nd, &err);
  if (st != DDI_OK) {
    set_error("ddi_plan_set_axes: %s", err.c_str());
    return st;
  }
  const double* n = nd.axis_n;
  const double* m = nd.axis_m;
  const double nm = (n[0] * m[0] + n[1] * m[1]) + n[2] * m[2];
  const double two_dv = 2.0 * p.dv;
  const unsigned blocks = (unsigned)((p.Mh + 255) / 256);
  if (p.prec == DDI_FP64)
    k_set_axes<double><<<blocks, 256, 0, s>>>(p.d_dirw, static_cast<double*>(p.d_scale), p.Mh, p.dim, n[0], n[1],
                                              n[2], m[0], m[1], m[2], nm, symbol_divisor(p.dim), two_dv);
  else
    k_set_axes<float><<<blocks, 256, 0, s>>>(p.d_dirw, static_cast<float*>(p.d_scale), p.Mh, p.dim, n[0], n[1],
                                             n[2], m[0], m[1], m[2], nm, symbol_divisor(p.dim), two_dv);
  DDI_LAUNCH_CHECK();
  for (int a = 0; a < 3; ++a) {
    p.desc.axis_n[a] = n[a];
    p.desc.axis_m[a] = m[a];
  }
  return DDI_OK;
}

void fill_info(const Plan& p, ddi_plan_info* info) {
  std::memset(info, 0, sizeof *info);
  info->dim = p.dim;
  info->precision = p.prec;
  for (int a = 0; a < 3; ++a) {
    info->n[a] = p.n[a];
    info->nf[a] = p.nf[a];
    info->tile[a] = p.tile[a];
  }
  info->width = p.w;
  info->beta = p.beta;
  info->nodes = p.M;
  info->nodes_used = p.Mh;
  info->spread_items = p.nunits;
  info->spread_split_tiles = p.nsplit;
  info->interp_items = (int)((p.Mh + 255) / 256);
  info->kmax = p.desc.kmax;
  info->nr = p.desc.nr;
  info->ntheta = p.desc.ntheta;
  info->nphi = p.desc.nphi;
  info->device_bytes = p.bytes;
  info->spread_tuned_ms = p.tuned_ms;
  info->split_k0 = p.split() ? p.desc.split_k0 : 0.0;
  info->ellipsoid = p.desc.ellipsoid;
  info->band[0] = p.band[0];
  info->band[1] = p.band[1];
  info->spread = p.spread_kind;
  info->yrange[0] = p.yr[0];
  info->yrange[1] = p.yr[1];
  if (p.spread_kind == DDI_SPREAD_COLUMNS) {
    info->tile[0] = kColX;
    info->tile[1] = p.dim == 3 ? kColY : p.nf[1];
    info->tile[2] = p.nf[2];
    info->spread_items = p.ncunits;
    info->spread_split_tiles = p.ncred;
  }
}

void destroy_plan(Plan& p) { free_plan(p); }

int take_nonfinite(Plan& p, cudaStream_t s) {
  int flag = 0;
  DDI_CUDA(cudaMemcpyAsync(&flag, p.d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, s));
  DDI_CUDA(cudaStreamSynchronize(s));
  if (!flag) return DDI_OK;
  DDI_CUDA(cudaMemsetAsync(p.d_nonfinite, 0, sizeof(int), s));
  set_error("the density held NaN or Inf");
  return DDI_ERR_NONFINITE;
}

}  // namespace ddi

// ==== C ABI ======================================================================================
using ddi::Plan;

extern "C" {

const char* ddi_status_str(int status) {
  switch (status) {
    case DDI_OK: return "DDI_OK";
    case DDI_ERR_ARG: return "DDI_ERR_ARG: invalid argument";
    case DDI_ERR_CUDA: return "DDI_ERR_CUDA: CUDA runtime error";
    case DDI_ERR_OOM: return "DDI_ERR_OOM: device allocation failed";
    case DDI_ERR_NONFINITE: return "DDI_ERR_NONFINITE: NaN or Inf encountered";
    case DDI_ERR_TIMEOUT: return "DDI_ERR_TIMEOUT: bounded device wait gave up";
    case DDI_ERR_NOCONV: return "DDI_ERR_NOCONV: iteration limit reached";
    case DDI_ERR_INTERNAL: return "DDI_ERR_INTERNAL: unexpected host-side failure";
    default: return "unknown ddi status";
  }
}

const char* ddi_last_error(void) { return ddi::last_error(); }

int ddi_quadrature_tables(const ddi_plan_desc* desc, int64_t* M, double* k, double* W, int32_t* l0) {
  return ddi::guarded("ddi_quadrature_tables", [&]() -> int {
    ddi_plan_desc d;
    std::string err;
    int s = ddi::normalise_desc(desc, &d, &err);
    if (s != DDI_OK) {
      ddi::set_error("%s", err.c_str());
      return s;
    }
    if (!M) {
      ddi::set_error("M must not be NULL");
      return DDI_ERR_ARG;
    }
    ddi::QuadTables t;
    ddi::build_quadrature(d, &t);
    *M = t.M;
    if (k) memcpy(k, t.k.data(), sizeof(double) * t.k.size());
    if (W) memcpy(W, t.W.data(), sizeof(double) * t.W.size());
    if (l0) {
      const int w = ddi::kernel_width(d);
      for (int64_t q = 0; q < t.M; ++q)
        for (int a = 0; a < d.dim; ++a)
          l0[d.dim * q + a] = (int32_t)ddi::fine_start(t.k[d.dim * q + a], t.h[a], 2 * d.n[a], w);
    }
    return DDI_OK;
  });
}

int ddi_plan_describe(const ddi_plan_desc* desc, ddi_plan_info* info) {
  return ddi::guarded("ddi_plan_describe", [&]() -> int {
    if (!info) {
      ddi::set_error("info must not be NULL");
      return DDI_ERR_ARG;
    }
    ddi_plan_desc d;
    std::string err;
    const int s = ddi::normalise_desc(desc, &d, &err);
    if (s != DDI_OK) {
      ddi::set_error("%s", err.c_str());
      return s;
    }
    std::memset(info, 0, sizeof *info);
    info->dim = d.dim;
    info->precision = d.precision;
    for (int a = 0; a < 3; ++a) {
      info->n[a] = a < d.dim ? d.n[a] : 1;
      info->nf[a] = a < d.dim ? 2 * d.n[a] : 1;
    }
    info->width = ddi::kernel_width(d);
    info->beta = ddi::kernel_beta(info->width);
    info->nodes = (int64_t)d.nr * d.ntheta * d.nphi;
    info->nodes_used = info->nodes / 2;
    info->kmax = d.kmax;
    info->nr = d.nr;
    info->ntheta = d.ntheta;
    info->nphi = d.nphi;
    info->split_k0 = d.split_k0 > 0.0 ? d.split_k0 : 0.0;
    info->ellipsoid = d.ellipsoid;
    ddi::split_band(d, info->width, info->band);
    return DDI_OK;
  });
}

int ddi_plan_create(ddi_plan* out, const ddi_plan_desc* desc, void* stream) {
  return ddi::guarded("ddi_plan_create", [&]() -> int {
    if (!out) {
      ddi::set_error("out is NULL");
      return DDI_ERR_ARG;
    }
    *out = nullptr;
    ddi_plan_s* h = new (std::nothrow) ddi_plan_s();
    if (!h) {
      ddi::set_error("host allocation failed");
      return DDI_ERR_OOM;
    }
    int s;
    try {
      s = ddi::create_plan(h->p, desc, static_cast<cudaStream_t>(stream));
      if (s == DDI_OK && desc->tile[0] < 0) s = ddi::tune_spread_tile(h->p, static_cast<cudaStream_t>(stream));
    } catch (...) {
      ddi::destroy_plan(h->p);  // what was allocated before the failure
      delete h;
      throw;
    }
    if (s != DDI_OK) {
      ddi::destroy_plan(h->p);
      delete h;
      return s;
    }
    *out = h;
    return DDI_OK;
  });
}

int ddi_plan_destroy(ddi_plan plan) {
  if (!plan) return DDI_OK;
  ddi::destroy_plan(plan->p);
  delete plan;
  return DDI_OK;
}

int ddi_plan_get_info(ddi_plan plan, ddi_plan_info* info) {
  if (!plan || !info) {
    ddi::set_error("plan and info must not be NULL");
    return DDI_ERR_ARG;
  }
  ddi::fill_info(plan->p, info);
  return DDI_OK;
}

int ddi_plan_set_axes(ddi_plan plan, const double* axis_n, const double* axis_m, void* stream) {
  return ddi::guarded("ddi_plan_set_axes", [&]() -> int {
    if (!plan || !axis_n) {
      ddi::set_error("ddi_plan_set_axes: plan and axis_n must not be NULL");
      return DDI_ERR_ARG;
    }
    return ddi::set_axes(plan->p, axis_n, axis_m, static_cast<cudaStream_t>(stream));
  });
}

int ddi_plan_node_order(ddi_plan plan, int64_t* q) {
  return ddi::guarded("ddi_plan_node_order", [&]() -> int {
    if (!plan || !q) {
      ddi::set_error("plan and q must not be NULL");
      return DDI_ERR_ARG;
    }
    memcpy(q, plan->p.order.data(), sizeof(int64_t) * plan->p.order.size());
    return DDI_OK;
  });
}

static int check_plan_ptrs(ddi_plan plan, const void* a, const void* b) {
  if (!plan || !a || !b) {
    ddi::set_error("plan and array pointers must not be NULL");
    return DDI_ERR_ARG;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->p.device) {
    ddi::set_error("the current device (%d) is not the plan's device (%d)", dev, plan->p.device);
    return DDI_ERR_ARG;
  }
  return DDI_OK;
}

int ddi_apply(ddi_plan plan, const void* rho, void* phi, void* stream) {
  return ddi::guarded("ddi_apply", [&]() -> int {
    DDI_TRY(check_plan_ptrs(plan, rho, phi));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan& p = plan->p;
    if (p.prec == DDI_FP64) {
      DDI_TRY(ddi::run_ddi<double>(p, static_cast<const double*>(rho), static_cast<double*>(phi), s));
    } else {
      DDI_TRY(ddi::run_ddi<float>(p, static_cast<const float*>(rho), static_cast<float*>(phi), s));
    }
    return p.desc.check_finite ? ddi::take_nonfinite(p, s) : DDI_OK;
  });
}

int ddi_plan_check(ddi_plan plan, void* stream) {
  return ddi::guarded("ddi_plan_check", [&]() -> int {
    if (!plan) {
      ddi::set_error("plan must not be NULL");
      return DDI_ERR_ARG;
    }
    return ddi::take_nonfinite(plan->p, static_cast<cudaStream_t>(stream));
  });
}

int ddi_apply_host(ddi_plan plan, const void* rho_host, void* phi_host, void* stream) {
  return ddi::guarded("ddi_apply_host", [&]() -> int {
    DDI_TRY(check_plan_ptrs(plan, rho_host, phi_host));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan& p = plan->p;
    const size_t bytes = p.real_size() * (size_t)p.grid_points();
    DDI_CUDA(cudaMemcpyAsync(p.d_io_in, rho_host, bytes, cudaMemcpyHostToDevice, s));
    if (p.prec == DDI_FP64) {
      DDI_TRY(ddi::run_ddi<double>(p, static_cast<const double*>(p.d_io_in), static_cast<double*>(p.d_io_out), s));
    } else {
      DDI_TRY(ddi::run_ddi<float>(p, static_cast<const float*>(p.d_io_in), static_cast<float*>(p.d_io_out), s));
    }
    DDI_CUDA(cudaMemcpyAsync(phi_host, p.d_io_out, bytes, cudaMemcpyDeviceToHost, s));
    return ddi::take_nonfinite(p, s);  // synchronises s
  });
}

int ddi_apply_timed(ddi_plan plan, const void* rho, void* phi, void* stream, const char** names, double* ms,
                    int cap, int* count) {
  return ddi::guarded("ddi_apply_timed", [&]() -> int {
    DDI_TRY(check_plan_ptrs(plan, rho, phi));
    if (!names || !ms || !count || cap < 1) {
      ddi::set_error("names, ms and count must not be NULL and cap >= 1");
      return DDI_ERR_ARG;
    }
    Plan& p = plan->p;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!p.ev_created) {
      for (cudaEvent_t& e : p.mark_ev) DDI_CUDA(cudaEventCreate(&e));
      p.ev_created = true;
    }
    p.timing = true;
    p.nmarks = 0;
    DDI_CUDA(cudaEventRecord(p.mark_ev[0], s));
    int st = p.prec == DDI_FP64
                 ? ddi::run_ddi<double>(p, static_cast<const double*>(rho), static_cast<double*>(phi), s)
                 : ddi::run_ddi<float>(p, static_cast<const float*>(rho), static_cast<float*>(phi), s);
    p.timing = false;
    if (st != DDI_OK) return st;
    DDI_CUDA(cudaStreamSynchronize(s));
    const int n = p.nmarks < cap ? p.nmarks : cap;
    for (int i = 0; i < n; ++i) {
      float t = 0.f;
      DDI_CUDA(cudaEventElapsedTime(&t, p.mark_ev[i], p.mark_ev[i + 1]));
      names[i] = p.mark_names[i];
      ms[i] = (double)t;
    }
    *count = n;
    return DDI_OK;
  });
}

int ddi_type2(ddi_plan plan, const void* rho, void* c, void* stream) {
  return ddi::guarded("ddi_type2", [&]() -> int {
    DDI_TRY(check_plan_ptrs(plan, rho, c));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan& p = plan->p;
    if (p.prec == DDI_FP64) {
      DDI_TRY(ddi::run_type2<double>(p, static_cast<const double*>(rho), s));
    } else {
      DDI_TRY(ddi::run_type2<float>(p, static_cast<const float*>(rho), s));
    }
    DDI_CUDA(cudaMemcpyAsync(c, p.d_c, p.cx_size() * p.Mh, cudaMemcpyDeviceToDevice, s));
    return DDI_OK;
  });
}

int ddi_type1(ddi_plan plan, const void* c, void* phi, void* stream) {
  return ddi::guarded("ddi_type1", [&]() -> int {
    DDI_TRY(check_plan_ptrs(plan, c, phi));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan& p = plan->p;
    DDI_CUDA(cudaMemcpyAsync(p.d_c, c, p.cx_size() * p.Mh, cudaMemcpyDeviceToDevice, s));
    if (p.prec == DDI_FP64) return ddi::run_type1_from_c<double>(p, static_cast<double*>(phi), s);
    return ddi::run_type1_from_c<float>(p, static_cast<float*>(phi), s);
  });
}

}  // extern "C"

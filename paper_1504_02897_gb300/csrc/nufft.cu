// NUFFT evaluation of the DDI quadrature sum (Sec. 2.1, Eq. DDI-Trun1).
//
//   Phi_j = Re sum_q W_q e^{i k_q.x_j} h^d sum_j' rho_j' e^{-i k_q.x_j'}
//
// With t_q = k_q h (per axis) and centred indices j' = j - n/2 the box centre cancels
// between the two transforms, so the path evaluates
//   f_q   = sum_j' rho_j' e^{-i t_q.j'}                         (type 2)
//   c_q   = 2 h^d W_q f_q       over one node of each (k, -k) pair
//   Phi_j = Re sum_q c_q e^{+i t_q.j'}                            (type 1)
// (the node set is closed under k -> -k with equal weights and rho is real, so the sum
// over the pair is twice the real part of one term).  Both transforms use a 2x
// oversampled grid and the exponential-of-semicircle kernel
//   psi(x) = exp(beta (sqrt(1 - (2x/w)^2) - 1)), |x| < w/2 (x in fine cells),
// with deconvolution by its Fourier transform psihat(2 pi j'/nf).  The nodes are fixed by
// the plan, so the per-axis kernel values psi_d(l - s_q) of every node are built once
// (FP64 on the host, rounded to the working precision) and read here.
//
// Launches (fft_nufft.cu holds the FFT passes):
//   forward FFT x (pad + deconvolution fused), y, z, pruned to the padded block
//   k_interp    one thread per node: f_q = sum over the w^d taps of psi F; writes
//               c_q = 2 h^d W_q f_q and c_q psi_z (the spread's per-plane factors)
//   k_spread    owner-computes spread over work units (tile, z-plane): a warp takes a
//               unit, streams the nodes whose taps reach that plane (ranges built by the
//               plan) and adds c psi_z psi_y psi_x into its shared-memory plane with plain
//               read-modify-writes (no other unit owns those cells); runs of nodes with
//               the same footprint are summed in registers first.  Every plane is
//               written once; long units are split into partial planes
//   k_reduce    sums the partial planes of split units
//   inverse FFT z, y, x (pruned to the cropped block; x fused with crop, deconvolution
//               and real part)
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace ddi {
namespace {

struct GridDims {
  int n[3];
  int nf[3];
};

GridDims dims_of(const Plan& p) {
  GridDims g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = p.n[d];
    g.nf[d] = p.nf[d];
  }
  return g;
}

// i in [0, 2 nf) -> i mod nf
__device__ __forceinline__ int wrap1(int i, int nf) { return i >= nf ? i - nf : i; }

// ---- interpolation (type 2) -----------------------------------------------------------------
template <typename T, int W, int DIM>
__global__ void __launch_bounds__(256)
    k_interp(const cx_t<T>* __restrict__ fine, const ushort4* __restrict__ l0, const T* __restrict__ psi,
             const T* __restrict__ scale, cx_t<T>* __restrict__ cout, cx_t<T>* __restrict__ czout,
             long long count, GridDims g) {
  using C = cx_t<T>;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const ushort4 s = l0[i];
  const T* ps = psi + i * 3 * W;
  T kx[W], ky[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    kx[a] = ps[a];
    ky[a] = ps[W + a];
  }
  T ar = 0, ai = 0;
  if (DIM == 3) {
#pragma unroll 1
    for (int az = 0; az < W; ++az) {
      const T wz = ps[2 * W + az];
      const long long zoff = (long long)wrap1(s.z + az, g.nf[2]) * g.nf[1];
      T zr = 0, zi = 0;
#pragma unroll
      for (int ay = 0; ay < W; ++ay) {
        const C* row = fine + (zoff + wrap1(s.y + ay, g.nf[1])) * g.nf[0];
        T rr = 0, ri = 0;
#pragma unroll
        for (int ax = 0; ax < W; ++ax) {
          const C v = __ldg(row + wrap1(s.x + ax, g.nf[0]));
          rr += kx[ax] * v.x;
          ri += kx[ax] * v.y;
        }
        zr += ky[ay] * rr;
        zi += ky[ay] * ri;
      }
      ar += wz * zr;
      ai += wz * zi;
    }
  } else {
#pragma unroll
    for (int ay = 0; ay < W; ++ay) {
      const C* row = fine + (long long)wrap1(s.y + ay, g.nf[1]) * g.nf[0];
      T rr = 0, ri = 0;
#pragma unroll
      for (int ax = 0; ax < W; ++ax) {
        const C v = __ldg(row + wrap1(s.x + ax, g.nf[0]));
        rr += kx[ax] * v.x;
        ri += kx[ax] * v.y;
      }
      ar += ky[ay] * rr;
      ai += ky[ay] * ri;
    }
  }
  const T sc = scale[i];
  const C c = cmk<C>(sc * ar, sc * ai);
  cout[i] = c;
  // factors of the spread's owned axis (z in 3D, y in 2D)
  const T* po = ps + (DIM == 3 ? 2 : 1) * W;
#pragma unroll
  for (int a = 0; a < W; ++a) czout[i * W + a] = cmk<C>(c.x * po[a], c.y * po[a]);
}

// c_q -> c_q psi_owned (the type-1 stage run on its own, from given node values)
template <typename T, int W, int DIM>
__global__ void k_expand(const cx_t<T>* __restrict__ c, const T* __restrict__ psi, cx_t<T>* __restrict__ czout,
                         long long count) {
  using C = cx_t<T>;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const C cq = c[i];
  const T* po = psi + i * 3 * W + (DIM == 3 ? 2 : 1) * W;
#pragma unroll
  for (int a = 0; a < W; ++a) czout[i * W + a] = cmk<C>(cq.x * po[a], cq.y * po[a]);
}

// ---- spreading (type 1) ------------------------------------------------------------------------
struct SpreadArgs {
  GridDims g;
  int tile[3];
  int ntile[3];
  const SpreadUnit* units;  // (tile, plane, visit range, slot), largest first
  int nunits;
  int* counter;             // next unit to take (zeroed before the launch)
  const int4* visits;       // (node, ox, oy, oz): starts relative to the tile origin
  const void* cz;           // [node][w] c psi_owned
  const void* psi;          // [node][3][w]
  void* fine;
  void* partial;            // [slot][plane cells]
};

// per-warp shared memory of k_spread: the owned plane and a stage of 32 nodes
template <typename T, int W>
struct alignas(16) WarpStage {
  T px[32][W];
  T py[32][W];
  cx_t<T> cz[32];
  int2 o[32];
};

// Spread, one warp per work unit = (tile, owned plane).  The plane's cells are touched by
// no other unit, so the warp accumulates them in its own shared-memory buffer with plain
// read-modify-writes and writes them once.  Persistent: warps take units from a counter
// (largest first).  Lanes stage 32 nodes at a time (kernel values along x and y, c psi
// along the owned axis, starts), then each node adds c psi_owned psi_y psi_x to the cells
// of its footprint in the plane (lanes: x fastest, then y rows).  Consecutive nodes with
// the same (oy, ox) are summed in registers and written once per run.  In 2D the owned
// plane is a y-row.
template <typename T, int W, int DIM>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(SpreadArgs a) {
  using C = cx_t<T>;
  constexpr int XL = W <= 8 ? 8 : 16;    // lanes along x
  constexpr int RL = 32 / XL;            // y rows per warp instruction (3D)
  constexpr int MR = (W + RL - 1) / RL;  // row iterations per (node, plane)
  constexpr int NM = DIM == 3 ? MR : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = a.tile[0], TY = a.tile[1], TZ = a.tile[2];
  const int RS = spread_row_stride(TX);
  const bool swz = spread_swizzle(TX);
  const int PSZ = DIM == 3 ? TY * RS : RS;  // cells of one plane buffer
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t per_warp = spread_warp_bytes(PSZ * sizeof(C), sizeof(WarpStage<T, W>));
  C* plane = reinterpret_cast<C*>(smem_raw + warp * per_warp);
  WarpStage<T, W>* stage = reinterpret_cast<WarpStage<T, W>*>(smem_raw + warp * per_warp + ((PSZ * sizeof(C) + 15) & ~(size_t)15));
  const int nfx = a.g.nf[0], nfy = a.g.nf[1], nfz = a.g.nf[2];
  const bool wrx = a.ntile[0] == 1, wry = a.ntile[1] == 1;
  const bool wrp = DIM == 3 ? a.ntile[2] == 1 : a.ntile[1] == 1;  // owned axis wraps in the tile
  const int nfp = DIM == 3 ? nfz : nfy;
  const int4* __restrict__ vis = a.visits;
  const C* __restrict__ czg = static_cast<const C*>(a.cz);
  const T* __restrict__ psi = static_cast<const T*>(a.psi);
  const int rx = lane % XL, ry = lane / XL;
  const int ncell = DIM == 3 ? TX * TY : TX;  // cells of one owned plane

  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(a.counter, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= a.nunits) break;
    const SpreadUnit U = a.units[u];
    for (int i = lane; i < PSZ; i += 32) plane[i] = cmk<C>((T)0, (T)0);
    __syncwarp();
    const int p = U.plane;
    T ar[NM], ai[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) ar[m] = ai[m] = (T)0;
    int run_x = INT_MIN, run_y = 0;
    C* cellp[NM];
    bool okp[NM];
    for (int kb = U.lo; kb < U.hi; kb += 32) {
      const int cnt = min(32, U.hi - kb);
      if (lane < cnt) {
        const int4 e = vis[kb + lane];
        const size_t node = (size_t)e.x;
        int az = p - (DIM == 3 ? e.w : e.z);
        if (wrp) az = az < 0 ? az + nfp : (az >= nfp ? az - nfp : az);
        const bool use = az >= 0 && az < W;
        stage->cz[lane] = use ? czg[node * W + az] : cmk<C>((T)0, (T)0);
        stage->o[lane] = make_int2(use ? e.y : INT_MIN + 1, e.z);
        const T* ps = psi + node * 3 * W;
#pragma unroll
        for (int q = 0; q < W; ++q) stage->px[lane][q] = ps[q];
        if (DIM == 3) {
#pragma unroll
          for (int q = 0; q < W; ++q) stage->py[lane][q] = ps[W + q];
        }
      }
      __syncwarp();
      for (int j = 0; j < cnt; ++j) {
        const int2 o = stage->o[j];
        if (o.x == INT_MIN + 1) continue;  // wrapping tiles only: this node misses plane p
        if (o.x != run_x || o.y != run_y) {
          if (run_x != INT_MIN) {
#pragma unroll
            for (int m = 0; m < NM; ++m)
              if (okp[m]) {
                C cur = *cellp[m];
                cur.x += ar[m];
                cur.y += ai[m];
                *cellp[m] = cur;
              }
#pragma unroll
            for (int m = 0; m < NM; ++m) ar[m] = ai[m] = (T)0;
          }
          // cells of this lane for the new footprint
          run_x = o.x;
          run_y = o.y;
          int xx = o.x + rx;
          if (wrx && xx < 0) xx += nfx;
          const bool okx = rx < W && (unsigned)xx < (unsigned)TX;
#pragma unroll
          for (int m = 0; m < NM; ++m) {
            const int r = ry + RL * m;
            int yy = o.y + r;
            if (wry && yy < 0) yy += nfy;
            okp[m] = okx && (DIM == 3 ? (r < W && (unsigned)yy < (unsigned)TY) : ry == 0);
            cellp[m] = plane + (DIM == 3 ? spread_cell(okp[m] ? yy : 0, okp[m] ? xx : 0, RS, swz) : (okp[m] ? xx : 0));
          }
        }
        const C czv = stage->cz[j];
        const T wx = rx < W ? stage->px[j][rx] : (T)0;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const int r = ry + RL * m;
          const T w = DIM == 3 ? (r < W ? stage->py[j][r] : (T)0) * wx : wx;
          ar[m] += czv.x * w;
          ai[m] += czv.y * w;
        }
      }
      __syncwarp();
    }
    if (run_x != INT_MIN) {
#pragma unroll
      for (int m = 0; m < NM; ++m)
        if (okp[m]) {
          C cur = *cellp[m];
          cur.x += ar[m];
          cur.y += ai[m];
          *cellp[m] = cur;
        }
    }
    __syncwarp();
    // write the plane (or this unit's partial plane)
    const int tx = U.tile % a.ntile[0];
    const int ty = (U.tile / a.ntile[0]) % a.ntile[1];
    const int tz = U.tile / (a.ntile[0] * a.ntile[1]);
    const int T0x = tile_origin(tx, TX, a.ntile[0], nfx);
    const int T0y = tile_origin(ty, TY, a.ntile[1], nfy);
    const int T0z = tile_origin(tz, TZ, a.ntile[2], nfz);
    if (U.slot < 0) {
      C* fine = static_cast<C*>(a.fine);
      for (int i = lane; i < ncell; i += 32) {
        const int lx = i % TX, ly = DIM == 3 ? i / TX : p;
        const int lz = DIM == 3 ? p : 0;
        const int gx = T0x + lx, gy = T0y + ly, gz = T0z + lz;
        const long long off =
            ((long long)(gz >= nfz ? gz - nfz : gz) * nfy + (gy >= nfy ? gy - nfy : gy)) * nfx + (gx >= nfx ? gx - nfx : gx);
        fine[off] = plane[DIM == 3 ? spread_cell(ly, lx, RS, swz) : lx];
      }
    } else {
      C* part = static_cast<C*>(a.partial) + (long long)U.slot * ncell;
      for (int i = lane; i < ncell; i += 32) {
        const int lx = i % TX, ly = i / TX;
        part[i] = plane[DIM == 3 ? spread_cell(ly, lx, RS, swz) : lx];
      }
    }
    __syncwarp();
  }
}

// Sums the partial planes of split units into the fine grid.
template <typename T, int DIM>
__global__ void k_reduce(const SplitUnit* __restrict__ split, const cx_t<T>* __restrict__ partial,
                         cx_t<T>* __restrict__ fine, GridDims g, int TX, int TY, int TZ, int ntx, int nty, int ntz) {
  using C = cx_t<T>;
  const SplitUnit st = split[blockIdx.x];
  const int ncell = DIM == 3 ? TX * TY : TX;
  const int tx = st.tile % ntx, ty = (st.tile / ntx) % nty, tz = st.tile / (ntx * nty);
  const int ox = tile_origin(tx, TX, ntx, g.nf[0]);
  const int oy = tile_origin(ty, TY, nty, g.nf[1]);
  const int oz = tile_origin(tz, TZ, ntz, g.nf[2]);
  for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
    T sr = 0, si = 0;
    for (int k = 0; k < st.nslots; ++k) {
      const C v = partial[(long long)(st.slot0 + k) * ncell + i];
      sr += v.x;
      si += v.y;
    }
    int gx = ox + i % TX;
    int gy = oy + (DIM == 3 ? i / TX : st.plane);
    int gz = oz + (DIM == 3 ? st.plane : 0);
    gx -= gx >= g.nf[0] ? g.nf[0] : 0;
    gy -= gy >= g.nf[1] ? g.nf[1] : 0;
    gz -= gz >= g.nf[2] ? g.nf[2] : 0;
    fine[((long long)gz * g.nf[1] + gy) * g.nf[0] + gx] = cmk<C>(sr, si);
  }
}

// ---- launch helpers ----------------------------------------------------------------------------
template <typename T, int W, int DIM>
int launch_interp(Plan& p, cudaStream_t s) {
  const long long cnt = p.Mh;
  k_interp<T, W, DIM><<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
      static_cast<const cx_t<T>*>(p.d_fine), static_cast<const ushort4*>(p.d_l0), static_cast<const T*>(p.d_psi),
      static_cast<const T*>(p.d_scale), static_cast<cx_t<T>*>(p.d_c), static_cast<cx_t<T>*>(p.d_cz), cnt,
      dims_of(p));
  DDI_LAUNCH_CHECK();
  return DDI_OK;
}

template <typename T, int W, int DIM>
int launch_expand(Plan& p, cudaStream_t s) {
  const long long cnt = p.Mh;
  k_expand<T, W, DIM><<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
      static_cast<const cx_t<T>*>(p.d_c), static_cast<const T*>(p.d_psi), static_cast<cx_t<T>*>(p.d_cz), cnt);
  DDI_LAUNCH_CHECK();
  return DDI_OK;
}

// launch geometry of the spread, fixed per plan (computed once so that applies make no
// host-side queries and can be recorded into a CUDA graph)
template <typename T, int W, int DIM>
int configure_spread(Plan& p, cudaStream_t) {
  const size_t plane_bytes = p.spread_plane_cells() * sizeof(cx_t<T>);
  const size_t smem = spread_warp_bytes(plane_bytes, sizeof(WarpStage<T, W>)) * (kSpreadThreads / 32);
  auto kern = k_spread<T, W, DIM>;
  {
    // the limit belongs to the kernel, shared by every plan (and thread): only raise it
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    DDI_CUDA(cudaFuncGetAttributes(&fa, kern));
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
      DDI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int per_sm = 0;
  DDI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSpreadThreads, smem));
  int sms = 0;
  DDI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device));
  p.spread_smem = smem;
  p.spread_blocks = std::max(1, std::min(per_sm * sms, (p.nunits + kSpreadThreads / 32 - 1) / (kSpreadThreads / 32)));
  return DDI_OK;
}

template <typename T, int W, int DIM>
int launch_spread(Plan& p, cudaStream_t s) {
  SpreadArgs a;
  a.g = dims_of(p);
  for (int d = 0; d < 3; ++d) {
    a.tile[d] = p.tile[d];
    a.ntile[d] = p.ntile[d];
  }
  a.units = p.d_units;
  a.nunits = p.nunits;
  a.counter = p.d_counter;
  a.visits = p.d_visits;
  a.cz = p.d_cz;
  a.psi = p.d_psi;
  a.fine = p.d_fine;
  a.partial = p.d_partial;
  auto kern = k_spread<T, W, DIM>;
  const size_t smem = p.spread_smem;
  const int blocks = p.spread_blocks;
  DDI_CUDA(cudaMemsetAsync(p.d_counter, 0, sizeof(int), s));
  kern<<<blocks, kSpreadThreads, smem, s>>>(a);
  DDI_LAUNCH_CHECK();
  p.mark("spread", s);
  if (p.nsplit > 0) {
    k_reduce<T, DIM><<<p.nsplit, 256, 0, s>>>(p.d_split, static_cast<const cx_t<T>*>(p.d_partial),
                                              static_cast<cx_t<T>*>(p.d_fine), dims_of(p), p.tile[0], p.tile[1],
                                              p.tile[2], p.ntile[0], p.ntile[1], p.ntile[2]);
    DDI_LAUNCH_CHECK();
    p.mark("spread_reduce", s);
  }
  return DDI_OK;
}

// kernel widths built per precision (the plan picks one of them from its tolerance)
#define DDI_WIDTH_SWITCH(FN)                                         \
  template <typename T, int DIM>                                    \
  int FN##_w(Plan& p, cudaStream_t s) {                             \
    if (sizeof(T) == 4) {                                           \
      switch (p.w) {                                                \
        case 6: return FN<T, 6, DIM>(p, s);                         \
        case 8: return FN<T, 8, DIM>(p, s);                         \
      }                                                             \
    } else {                                                        \
      switch (p.w) {                                                \
        case 10: return FN<T, 10, DIM>(p, s);                       \
        case 12: return FN<T, 12, DIM>(p, s);                       \
        case 14: return FN<T, 14, DIM>(p, s);                       \
        case 16: return FN<T, 16, DIM>(p, s);                       \
      }                                                             \
    }                                                               \
    set_error("kernel width %d not built for this precision", p.w); \
    return DDI_ERR_ARG;                                             \
  }

DDI_WIDTH_SWITCH(launch_interp)
DDI_WIDTH_SWITCH(launch_expand)
DDI_WIDTH_SWITCH(launch_spread)
DDI_WIDTH_SWITCH(configure_spread)

}  // namespace

int configure_kernels(Plan& p) {
  if (p.prec == DDI_FP64)
    return p.dim == 3 ? configure_spread_w<double, 3>(p, nullptr) : configure_spread_w<double, 2>(p, nullptr);
  return p.dim == 3 ? configure_spread_w<float, 3>(p, nullptr) : configure_spread_w<float, 2>(p, nullptr);
}

// Device time of the spread (and its partial-plane reduction) for the plan's current
// tile: the best of `reps` timed launches after one untimed one, on zeroed node values
// (the cost depends on the node set and the tile, not on the values).
int time_spread(Plan& p, cudaStream_t s, int reps, float* ms) {
  DDI_CUDA(cudaMemsetAsync(p.d_cz, 0, p.cx_size() * (size_t)p.Mh * p.w, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    set_error("time_spread: %s", cudaGetErrorString(cudaGetLastError()));
    return DDI_ERR_CUDA;
  }
  auto once = [&]() {
    if (p.prec == DDI_FP64) return p.dim == 3 ? launch_spread_w<double, 3>(p, s) : launch_spread_w<double, 2>(p, s);
    return p.dim == 3 ? launch_spread_w<float, 3>(p, s) : launch_spread_w<float, 2>(p, s);
  };
  int st = once();
  float best = 0.f;
  for (int r = 0; r < reps && st == DDI_OK; ++r) {
    cudaEventRecord(e0, s);
    st = once();
    cudaEventRecord(e1, s);
    float t = 0.f;
    if (st == DDI_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) {
      if (r == 0 || t < best) best = t;
    } else if (st == DDI_OK) {
      set_error("time_spread: %s", cudaGetErrorString(cudaGetLastError()));
      st = DDI_ERR_CUDA;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return st;
}

template <typename T>
int run_type2(Plan& p, const T* rho, cudaStream_t s) {
  DDI_TRY(nufft_forward_fft<T>(p, rho, s));
  DDI_TRY((p.dim == 3 ? launch_interp_w<T, 3>(p, s) : launch_interp_w<T, 2>(p, s)));
  p.mark("interp", s);
  return DDI_OK;
}

template <typename T>
int run_type1(Plan& p, T* phi, cudaStream_t s) {
  DDI_TRY((p.dim == 3 ? launch_spread_w<T, 3>(p, s) : launch_spread_w<T, 2>(p, s)));
  return nufft_inverse_fft<T>(p, phi, s);
}

template <typename T>
int run_type1_from_c(Plan& p, T* phi, cudaStream_t s) {
  DDI_TRY((p.dim == 3 ? launch_expand_w<T, 3>(p, s) : launch_expand_w<T, 2>(p, s)));
  return run_type1<T>(p, phi, s);
}

template <typename T>
int run_ddi(Plan& p, const T* rho, T* phi, cudaStream_t s) {
  DDI_TRY(run_type2<T>(p, rho, s));
  return run_type1<T>(p, phi, s);
}

template int run_type2<float>(Plan&, const float*, cudaStream_t);
template int run_type2<double>(Plan&, const double*, cudaStream_t);
template int run_type1_from_c<float>(Plan&, float*, cudaStream_t);
template int run_type1_from_c<double>(Plan&, double*, cudaStream_t);
template int run_ddi<float>(Plan&, const float*, float*, cudaStream_t);
template int run_ddi<double>(Plan&, const double*, double*, cudaStream_t);

}  // namespace ddi

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
//   k_interp    8 (w <= 8) or 16 lanes per node: f_q = sum over the w^d taps of psi F,
//               each footprint row read as one contiguous segment; writes
//               c_q = 2 h^d W_q f_q
//   k_spread    owner-computes spread over work units (tile, z-plane in 3D; tile in
//               2D): a warp takes a unit, streams the nodes whose taps reach that plane
//               (ranges built by the plan) and adds c psi_z psi_y psi_x into its
//               shared-memory plane with plain read-modify-writes (no other unit owns
//               those cells).  Every plane is written once; long units are split into
//               partial planes
//   k_reduce    sums the partial planes of split units
//   inverse FFT z, y, x (pruned to the cropped block; x fused with crop, deconvolution
//               and real part)
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <mutex>
#include <utility>

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

// kernel values of one axis of a node (w contiguous values), in 16- or 8-byte loads
template <typename T, int W>
__device__ __forceinline__ void load_taps(const T* __restrict__ src, T (&dst)[W]) {
  if constexpr (sizeof(T) == 4 && W % 4 == 0) {
#pragma unroll
    for (int k = 0; k < W / 4; ++k) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src) + k);
      dst[4 * k] = v.x;
      dst[4 * k + 1] = v.y;
      dst[4 * k + 2] = v.z;
      dst[4 * k + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 4 && W % 2 == 0) {
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(src) + k);
      dst[2 * k] = v.x;
      dst[2 * k + 1] = v.y;
    }
  } else if constexpr (sizeof(T) == 8 && W % 2 == 0) {
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(src) + k);
      dst[2 * k] = v.x;
      dst[2 * k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) dst[k] = __ldg(src + k);
  }
}

// ---- interpolation (type 2) -----------------------------------------------------------------
// XL lanes per node (one x tap each; 8 for w <= 8, else 16), 32 / XL nodes per warp: the
// lanes of a node read each footprint row of the fine grid as one contiguous segment,
// accumulate the psi_y (and psi_z) weighted sums in registers, and the node's value is
// the psi_x-weighted sum over its lanes (shuffle reduction).
// (at most 64 registers in FP32, so that 4 CTAs per SM keep enough loads in flight)
template <typename T, int W, int DIM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
    k_interp(const cx_t<T>* __restrict__ fine, const ushort4* __restrict__ l0, const T* __restrict__ psi,
             const T* __restrict__ scale, cx_t<T>* __restrict__ cout, long long count, GridDims g) {
  using C = cx_t<T>;
  constexpr int XL = W <= 8 ? 8 : 16;
  const int lane = threadIdx.x & 31;
  const int rx = lane % XL;
  const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / XL;
  const bool valid = i0 < count;  // lanes past the end compute a copy of the last node
  const long long i = valid ? i0 : count - 1;
  const ushort4 s = l0[i];
  const T* ps = psi + i * 3 * W;
  T ky[W], kz[W];
  load_taps<T, W>(ps + W, ky);
  if (DIM == 3) load_taps<T, W>(ps + 2 * W, kz);
  const bool on = rx < W;
  const T kx = on ? __ldg(ps + rx) : (T)0;
  const int xx = wrap1(s.x + (on ? rx : 0), g.nf[0]);
  int yoff[W];  // row offsets within a plane (a plane holds < 2^31 cells)
#pragma unroll
  for (int ay = 0; ay < W; ++ay) yoff[ay] = wrap1(s.y + ay, g.nf[1]) * g.nf[0];
  T ar = 0, ai = 0;
  if (DIM == 3) {
    const long long plane = (long long)g.nf[1] * g.nf[0];
#pragma unroll
    for (int az = 0; az < W; ++az) {
      const C* zp = fine + wrap1(s.z + az, g.nf[2]) * plane + xx;
      T zr = 0, zi = 0;
#pragma unroll
      for (int ay = 0; ay < W; ++ay) {
        const C v = __ldg(zp + yoff[ay]);
        zr += ky[ay] * v.x;
        zi += ky[ay] * v.y;
      }
      ar += kz[az] * zr;
      ai += kz[az] * zi;
    }
  } else {
#pragma unroll
    for (int ay = 0; ay < W; ++ay) {
      const C v = __ldg(fine + xx + yoff[ay]);
      ar += ky[ay] * v.x;
      ai += ky[ay] * v.y;
    }
  }
  ar *= kx;
  ai *= kx;
#pragma unroll
  for (int o = XL / 2; o > 0; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
  }
  if (rx == 0 && valid) {
    const T sc = scale[i];
    cout[i] = cmk<C>(sc * ar, sc * ai);
  }
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
  const void* c;            // [node] c_q
  const void* psi;          // [node][3][w]
  void* fine;
  void* partial;            // [slot][TY][TX]
};

// per-warp shared memory of k_spread: the plane buffer and a stage of 32 nodes
template <typename T>
struct alignas(16) NodeHead {
  cx_t<T> cz;     // c_q psi_z(plane) (3D), c_q (2D)
  int base;       // buffer index of the footprint's first cell
  unsigned mask;  // taps inside the tile: bit t (x tap t), bit 16 + t (y tap t)
};
template <typename T, int W>
struct alignas(16) WarpStage {
  static constexpr int XL = W <= 8 ? 8 : 16, RL = 32 / XL, MR = (W + RL - 1) / RL, PW = MR * RL;
  T px[32][W];
  T py[32][PW];  // psi_y regrouped per lane row: py[j][MR r + m] = psi_y(r + RL m), 0 past w
  NodeHead<T> hd[32];
};
static_assert(sizeof(WarpStage<float, 8>) == spread_stage_bytes(8, 4), "stage size");
static_assert(sizeof(WarpStage<float, 6>) == spread_stage_bytes(6, 4), "stage size");
static_assert(sizeof(WarpStage<double, 14>) == spread_stage_bytes(14, 8), "stage size");
static_assert(sizeof(WarpStage<double, 10>) == spread_stage_bytes(10, 8), "stage size");

// taps t in [0, w) of a footprint starting at o that land inside [0, T), as a bit mask
__device__ __forceinline__ unsigned tap_mask(int o, int T, int w) {
  const int lo = o < 0 ? -o : 0;
  const int hi = T - o < w ? T - o : w;
  if (hi <= lo) return 0u;
  return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

// Spread, one warp per work unit.  A unit is a (tile, z-plane) in 3D and a whole tile in
// 2D: a plane of TY x TX fine cells that no other unit writes, so the warp accumulates it
// in its own shared-memory buffer with plain read-modify-writes and writes it once.
// Persistent: warps take units from a counter (largest first).  Lanes stage 32 nodes at a
// time (kernel values along x and y, c_q psi_z(plane), the footprint's first cell and the
// mask of its taps inside the tile), then the warp adds each node's w x w footprint
// c psi_y psi_x into the plane: lanes are (x, row) pairs, XL along x and 32/XL rows per
// instruction.  Long units are split into pieces that write partial planes (k_reduce).
template <typename T, int W, int DIM>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(SpreadArgs a) {
  using C = cx_t<T>;
  using S = WarpStage<T, W>;
  constexpr int XL = S::XL, RL = S::RL, MR = S::MR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = a.tile[0], TY = a.tile[1], TZ = a.tile[2];
  const int RS = spread_row_stride(TX);
  const int PSZ = TY * RS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t per_warp = spread_warp_bytes(PSZ * sizeof(C), sizeof(S));
  C* plane = reinterpret_cast<C*>(smem_raw + warp * per_warp);
  S* stage = reinterpret_cast<S*>(smem_raw + warp * per_warp + ((PSZ * sizeof(C) + 15) & ~(size_t)15));
  const int nfx = a.g.nf[0], nfy = a.g.nf[1], nfz = a.g.nf[2];
  // an axis held by a single tile wraps around inside it
  const bool wrx = a.ntile[0] == 1, wry = a.ntile[1] == 1, wrz = DIM == 3 && a.ntile[2] == 1;
  const bool wrap = wrx || wry;
  const int4* __restrict__ vis = a.visits;
  const C* __restrict__ cg = static_cast<const C*>(a.c);
  const T* __restrict__ psi = static_cast<const T*>(a.psi);
  const int rx = lane % XL, ry = lane / XL;
  const int rxc = rx < W ? rx : W - 1;
  // this lane's cell of the footprint per row iteration: required mask bits, buffer offset
  unsigned lbit[MR];
  int loff[MR];
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int r = ry + RL * m;
    lbit[m] = (rx < W && r < W) ? ((1u << rx) | (1u << (16 + r))) : 0xFFFFFFFFu;
    loff[m] = r * RS + rx;
  }

  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(a.counter, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= a.nunits) break;
    const SpreadUnit U = a.units[u];
    for (int i = lane; i < PSZ; i += 32) plane[i] = cmk<C>((T)0, (T)0);
    __syncwarp();
    const int p = U.plane;
    for (int kb = U.lo; kb < U.hi; kb += 32) {
      const int cnt = min(32, U.hi - kb);
      if (lane < cnt) {
        const int4 e = vis[kb + lane];
        const size_t node = (size_t)e.x;
        const T* ps = psi + node * 3 * W;
        bool use = true;
        T pz = (T)1;
        if (DIM == 3) {
          int az = p - e.w;
          if (wrz) az = az < 0 ? az + nfz : (az >= nfz ? az - nfz : az);
          use = az >= 0 && az < W;
          pz = use ? ps[2 * W + az] : (T)0;
        }
        const C cq = cg[node];
        T tx[W], ty[W];
        load_taps<T, W>(ps, tx);
        load_taps<T, W>(ps + W, ty);
        const unsigned xm = wrx ? (1u << W) - 1u : tap_mask(e.y, TX, W);
        const unsigned ym = wry ? (1u << W) - 1u : tap_mask(e.z, TY, W);
        NodeHead<T> h;
        h.cz = cmk<C>(cq.x * pz, cq.y * pz);
        h.base = e.z * RS + e.y;
        h.mask = use ? (xm | (ym << 16)) : 0u;
        stage->hd[lane] = h;
#pragma unroll
        for (int q = 0; q < W; ++q) stage->px[lane][q] = tx[q];
#pragma unroll
        for (int r = 0; r < RL; ++r)
#pragma unroll
          for (int m = 0; m < MR; ++m) stage->py[lane][MR * r + m] = r + RL * m < W ? ty[r + RL * m] : (T)0;
      }
      __syncwarp();
      if (!wrap) {
        for (int j = 0; j < cnt; ++j) {
          const NodeHead<T> h = stage->hd[j];
          const T wx = stage->px[j][rxc];
          T wy[MR];
#pragma unroll
          for (int m = 0; m < MR; ++m) wy[m] = stage->py[j][MR * ry + m];
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            if ((h.mask & lbit[m]) == lbit[m]) {
              const T w = wy[m] * wx;
              C* cell = plane + h.base + loff[m];
              C v = *cell;
              v.x += h.cz.x * w;
              v.y += h.cz.y * w;
              *cell = v;
            }
          }
          __syncwarp();  // the next node's cells may belong to other lanes
        }
      } else {
        for (int j = 0; j < cnt; ++j) {
          const NodeHead<T> h = stage->hd[j];
          if (h.mask == 0u) continue;  // this node misses plane p (uniform over the warp)
          const int4 e = vis[kb + j];
          const T wx = stage->px[j][rxc];
          int xx = e.y + rx;
          if (wrx && xx < 0) xx += nfx;
          const bool okx = rx < W && (unsigned)xx < (unsigned)TX;
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            const int r = ry + RL * m;
            int yy = e.z + r;
            if (wry && yy < 0) yy += nfy;
            if (okx && r < W && (unsigned)yy < (unsigned)TY) {
              const T w = stage->py[j][MR * ry + m] * wx;
              C* cell = plane + yy * RS + xx;
              C v = *cell;
              v.x += h.cz.x * w;
              v.y += h.cz.y * w;
              *cell = v;
            }
          }
          __syncwarp();
        }
      }
      __syncwarp();
    }
    __syncwarp();
    // write the plane (or this unit's partial plane)
    const int tx = U.tile % a.ntile[0];
    const int ty = (U.tile / a.ntile[0]) % a.ntile[1];
    const int tz = U.tile / (a.ntile[0] * a.ntile[1]);
    if (U.slot < 0) {
      const int T0x = tile_origin(tx, TX, a.ntile[0], nfx);
      const int T0y = tile_origin(ty, TY, a.ntile[1], nfy);
      int gz = DIM == 3 ? tile_origin(tz, TZ, a.ntile[2], nfz) + p : 0;
      gz -= gz >= nfz ? nfz : 0;
      C* fine = static_cast<C*>(a.fine) + (long long)gz * nfy * nfx;
      for (int ly = 0; ly < TY; ++ly) {
        int gy = T0y + ly;
        gy -= gy >= nfy ? nfy : 0;
        for (int lx = lane; lx < TX; lx += 32) {
          int gx = T0x + lx;
          gx -= gx >= nfx ? nfx : 0;
          fine[(long long)gy * nfx + gx] = plane[ly * RS + lx];
        }
      }
    } else {
      C* part = static_cast<C*>(a.partial) + (long long)U.slot * TX * TY;
      for (int ly = 0; ly < TY; ++ly)
        for (int lx = lane; lx < TX; lx += 32) part[ly * TX + lx] = plane[ly * RS + lx];
    }
    __syncwarp();
  }
}

// Sums the partial planes of split units into the fine grid: one thread per (split unit,
// cell), blockIdx.y = split unit - split0, partials summed in slot order (deterministic).
template <typename T, int DIM>
__global__ void __launch_bounds__(256)
    k_reduce(const SplitUnit* __restrict__ split, const cx_t<T>* __restrict__ partial, cx_t<T>* __restrict__ fine,
             GridDims g, int TX, int TY, int TZ, int ntx, int nty, int ntz, int split0) {
  using C = cx_t<T>;
  const int ncell = TX * TY;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell) return;
  const SplitUnit st = split[split0 + blockIdx.y];
  const int tx = st.tile % ntx, ty = (st.tile / ntx) % nty, tz = st.tile / (ntx * nty);
  const C* src = partial + (long long)st.slot0 * ncell + i;
  T sr = 0, si = 0;
  int k = 0;
  for (; k + 4 <= st.nslots; k += 4) {
    C v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __ldg(src + (long long)(k + q) * ncell);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sr += v[q].x;
      si += v[q].y;
    }
  }
  for (; k < st.nslots; ++k) {
    const C v = __ldg(src + (long long)k * ncell);
    sr += v.x;
    si += v.y;
  }
  int gx = tile_origin(tx, TX, ntx, g.nf[0]) + i % TX;
  int gy = tile_origin(ty, TY, nty, g.nf[1]) + i / TX;
  int gz = (DIM == 3 ? tile_origin(tz, TZ, ntz, g.nf[2]) : 0) + (DIM == 3 ? st.plane : 0);
  gx -= gx >= g.nf[0] ? g.nf[0] : 0;
  gy -= gy >= g.nf[1] ? g.nf[1] : 0;
  gz -= gz >= g.nf[2] ? g.nf[2] : 0;
  fine[((long long)gz * g.nf[1] + gy) * g.nf[0] + gx] = cmk<C>(sr, si);
}

// ---- column spreading (type 1, FP32 3D) -------------------------------------------------------
// A warp owns one column of kColX x kColY = 8 x 8 fine cells in x-y (lane (lx, ly) holds the
// cells (lx, ly) and (lx, ly + 4)) and W of its z-planes in registers: plane p (absolute,
// unwrapped) lives in acc0/acc1[p mod W].  It streams the unit's visits in order of their
// first z tap s: while zb < s the plane zb is complete (no later visit reaches it), so it
// is written out and its registers cleared for plane zb + W.
// Nodes with the same first z tap and the same psi_z row (a z class: one quadrature ring
// has a single k_z) are consecutive in a column's list.  For such a run the lane first sums
// g = sum c_q psi_x(x - l0x) psi_y(y - l0y) (one packed FP32 FMA per node and cell), then
// adds g psi_z(p - s) to the W planes p = s .. s + W - 1 once: c psi_x psi_y psi_z summed in
// the order (node, then z) instead of W products per node, exact up to rounding order.
// psi_x psi_y is 0 outside the footprint.  No shared-memory read-modify-write and no
// atomics: each cell belongs to one lane.
// Nodes are staged NS at a time in the warp's shared memory: psi_z in rotated order, each
// value twice (entry k holds plane k mod W of the node's window, so the add loop is the same
// for every node and registers never move), psi_x and psi_y in zero-padded rows (a lane's
// tap index needs no bounds test), and a header (first z tap with the run-start flag, byte
// offsets of the node's psi_x / psi_y entries for the column's first cell, c_q).
// Planes that several units touch go to partial slots (each such plane's slots are
// contiguous, in unit order) that k_reduce_col sums in order (deterministic).  Planes
// written directly use streaming stores, so they do not push the partial slots out of L2
// before the reduction reads them.
//
// Row strides (words) are 4 mod 8, so the 16-byte stores of 8 consecutive lanes (each
// writing its own node's row) fall in 8 distinct bank quadruples: conflict-free staging.
static_assert(kColX == 8 && kColY == 8, "lane (lx, ly) holds cells (lx, ly) and (lx, ly + 4) of an 8 x 8 column");
constexpr int kColThreads = 128;  // 4 warps per CTA, each taking units on its own
template <int W, int NS>
struct alignas(16) ColStage {
  static constexpr int PZ = ((2 * W + 7) / 8) * 8 + 4;  // psi_z, rotated, each value twice, then padding
  static constexpr int PX = ((W + 15 + 7) / 8) * 8 + 4;  // psi at [8, 8 + W): index c + 8 - o, c in [0, 8), o in [1-W, 8)
  float pz[NS][PZ];
  float px[NS][PX];
  float py[NS][PX];
  int4 hd[NS];  // byte offsets of px[j][8 - ox] and py[j][8 - oy]; c_q (two floats)
  int sz[NS];   // first z tap
};

struct ColArgs {
  int nf[3];
  int ncx;
  const ColUnit* units;
  int nunits;
  int* counter;
  const int2* visits;
  const float2* c;
  const float* psi;  // [node][3][w]
  float2* fine;
  float2* partial;        // [slot][kColY * kColX]
  const int* unit_slots;  // per unit: the partial slot of each leading, then trailing plane
};

// a += x with the rounding error of the sum carried in c (compensated summation, Kahan):
// y = x - c, t = a + y, c = (t - a) - y, a = t
__device__ __forceinline__ void kahan_add2(float2& a, float2& c, float2 x) {
  const float2 y = __fadd2_rn(x, make_float2(-c.x, -c.y));
  const float2 t = __fadd2_rn(a, y);
  c = __fadd2_rn(__fadd2_rn(t, make_float2(-a.x, -a.y)), make_float2(-y.x, -y.y));
  a = t;
}

// acc_k += g psi_z(k) for the run whose rotated, doubled psi_z row is pz; COMP: compensated
template <int W, bool COMP>
__device__ __forceinline__ void col_apply(float2 (&acc0)[W], float2 (&acc1)[W], float2 (&cmp0)[W], float2 (&cmp1)[W],
                                          const float* pz, float2 g0, float2 g1) {
  const float2* p2 = reinterpret_cast<const float2*>(pz);
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const float2 v = p2[k];
    if constexpr (COMP) {
      kahan_add2(acc0[k], cmp0[k], __fmul2_rn(g0, v));
      kahan_add2(acc1[k], cmp1[k], __fmul2_rn(g1, v));
    } else {
      acc0[k] = __ffma2_rn(g0, v, acc0[k]);
      acc1[k] = __ffma2_rn(g1, v, acc1[k]);
    }
  }
}

#define DDI_COL_CASES(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15)

template <int W, int NS, bool COMP>
__global__ void __launch_bounds__(kColThreads) k_spread_col(ColArgs a) {
  using S = ColStage<W, NS>;
  static_assert(W <= 16, "planes 0..15 of the window");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  S* st = reinterpret_cast<S*>(smem_raw) + warp;
  const int lx = lane & 7, ly = lane >> 3;
  const int lx4 = 4 * lx, ly4 = 4 * ly;
  const int nfx = a.nf[0], nfz = a.nf[2];
  const long long plane = (long long)nfx * a.nf[1];
  const unsigned st_off = (unsigned)(reinterpret_cast<unsigned char*>(st) - smem_raw);
  // the zero padding of the psi_x / psi_y rows never changes: written once
  for (int i = lane; i < NS * S::PX; i += 32) {
    (&st->px[0][0])[i] = 0.f;
    (&st->py[0][0])[i] = 0.f;
  }
  __syncwarp();
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(a.counter, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= a.nunits) break;
    const ColUnit U = a.units[u];
    const int cx = U.col % a.ncx, cy = U.col / a.ncx;
    const long long cell = (long long)(cy * kColY + ly) * nfx + cx * kColX + lx;  // cell (lx, ly); + 4 nfx: (lx, ly + 4)
    const int zpart_hi = U.z1 - U.phi;
    float2 acc0[W], acc1[W], cmp0[W], cmp1[W];
#pragma unroll
    for (int k = 0; k < W; ++k) acc0[k] = acc1[k] = cmp0[k] = cmp1[k] = make_float2(0.f, 0.f);
    int zb = U.z0;
    // write plane zb (direct, or a partial slot when other units touch it), clear its registers
    auto flush = [&]() {
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      switch (zb % W) {
#define DDI_TAKE(R)                                                  \
  case R:                                                            \
    if constexpr (R < W) {                                           \
      v0 = COMP ? __fadd2_rn(acc0[R], make_float2(-cmp0[R].x, -cmp0[R].y)) : acc0[R]; \
      v1 = COMP ? __fadd2_rn(acc1[R], make_float2(-cmp1[R].x, -cmp1[R].y)) : acc1[R]; \
      acc0[R] = acc1[R] = cmp0[R] = cmp1[R] = make_float2(0.f, 0.f); \
    }                                                                \
    break;
        DDI_COL_CASES(DDI_TAKE)
#undef DDI_TAKE
      }
      const int r = zb - U.z0;
      if (r < U.plo || zb >= zpart_hi) {
        const int k = r < U.plo ? r : U.plo + (zb - zpart_hi);
        float2* dst = a.partial + (size_t)__ldg(a.unit_slots + U.slot0 + k) * (kColX * kColY) + lane;
        dst[0] = v0;
        dst[32] = v1;
      } else {
        float2* dst = a.fine + (zb >= nfz ? zb - nfz : zb) * plane + cell;
        __stcs(dst, v0);
        __stcs(dst + 4 * nfx, v1);
      }
      ++zb;
    };
    for (int kb = U.lo; kb < U.hi; kb += NS) {
      const int cnt = min(NS, U.hi - kb);
      bool run_start = false;
      if (lane < cnt) {
        // one axis at a time, each stored as soon as it arrives (few registers live beside
        // the accumulators)
        const int2 v = a.visits[kb + lane];
        run_start = (v.y >> 12) & 1;
        const float* ps = a.psi + (size_t)v.x * 3 * W;
        {
          float t[W];
          load_taps<float, W>(ps, t);
#pragma unroll
          for (int k = 0; k < W; ++k) st->px[lane][8 + k] = t[k];
        }
        {
          float t[W];
          load_taps<float, W>(ps + W, t);
#pragma unroll
          for (int k = 0; k < W; ++k) st->py[lane][8 + k] = t[k];
        }
        const int sz = v.y >> 13;
        {
          float t[W];
          load_taps<float, W>(ps + 2 * W, t);
          float2* pzr = reinterpret_cast<float2*>(st->pz[lane]);
          const int rot = sz % W;  // tap dz feeds plane s + dz, held in register (s + dz) mod W
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const int q = rot + k < W ? rot + k : rot + k - W;
            pzr[q] = make_float2(t[k], t[k]);
          }
        }
        const float2 cq = __ldg(a.c + v.x);
        const int ox = (v.y & 63) - 16, oy = ((v.y >> 6) & 63) - 16;
        const unsigned pxo = st_off + (unsigned)(offsetof(S, px) + (lane * S::PX + 8 - ox) * sizeof(float));
        const unsigned pyo = st_off + (unsigned)(offsetof(S, py) + (lane * S::PX + 8 - oy) * sizeof(float));
        st->hd[lane] = make_int4((int)pxo, (int)pyo, __float_as_int(cq.x), __float_as_int(cq.y));
        st->sz[lane] = sz;
      }
      // runs of one z class: bit j set where staged visit j starts one (visit 0 always starts
      // the batch's first run, which may continue a run of the previous batch)
      unsigned starts = __ballot_sync(0xffffffffu, run_start) | 1u;
      __syncwarp();
      while (starts) {
        const int j0 = __ffs(starts) - 1;
        starts &= starts - 1;
        const int j1 = starts ? __ffs(starts) - 1 : cnt;
        const int sr = st->sz[j0];
        while (zb < sr) flush();
        // g: the run's sum of c psi_x psi_y per cell, then added to the W planes with psi_z
        float2 g0 = make_float2(0.f, 0.f), g1 = g0;
#pragma unroll 2
        for (int j = j0; j < j1; ++j) {
          const int4 h = st->hd[j];
          const float wx = *reinterpret_cast<const float*>(smem_raw + h.x + lx4);
          const float* py = reinterpret_cast<const float*>(smem_raw + h.y + ly4);
          const float w0 = wx * py[0], w1 = wx * py[4];
          const float2 cq = make_float2(__int_as_float(h.z), __int_as_float(h.w));
          g0 = __ffma2_rn(make_float2(w0, w0), cq, g0);
          g1 = __ffma2_rn(make_float2(w1, w1), cq, g1);
        }
        col_apply<W, COMP>(acc0, acc1, cmp0, cmp1, st->pz[j0], g0, g1);
      }
      __syncwarp();
    }
    while (zb < U.z1) flush();
  }
}

// Planes of a column that several units touch: one warp per entry, a lane per two cells;
// the entry's partial slots are contiguous (s0 .. s0 + ns - 1, in unit order) and summed in
// that order (deterministic), eight loads in flight at a time.
__global__ void __launch_bounds__(256)
    k_reduce_col(const ColRed* __restrict__ red, int nred, const float2* __restrict__ partial,
                 float2* __restrict__ fine, int nfx, int nfy, int ncx) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= nred) return;
  const int lane = threadIdx.x & 31;
  const int4 r = __ldg(reinterpret_cast<const int4*>(red) + e);  // col, z, s0, ns
  const float4* src = reinterpret_cast<const float4*>(partial + (size_t)r.z * (kColX * kColY)) + lane;
  // lane: cells 2 lane and 2 lane + 1 of the slot (row-major 8 x 8)
  float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
  int k = 0;
  for (; k + 8 <= r.w; k += 8) {
    float4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcs(src + (size_t)(k + q) * (kColX * kColY / 2));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sum.x += v[q].x;
      sum.y += v[q].y;
      sum.z += v[q].z;
      sum.w += v[q].w;
    }
  }
  for (; k < r.w; ++k) {
    const float4 v = __ldcs(src + (size_t)k * (kColX * kColY / 2));
    sum.x += v.x;
    sum.y += v.y;
    sum.z += v.z;
    sum.w += v.w;
  }
  const int cx = r.x % ncx, cy = r.x / ncx;
  const int c0 = 2 * lane;  // row c0 / 8, columns c0 % 8 and c0 % 8 + 1
  const long long cell = (long long)(cy * kColY + c0 / 8) * nfx + cx * kColX + c0 % 8;
  *reinterpret_cast<float4*>(fine + (long long)r.y * nfx * nfy + cell) = sum;
}

// 2D column spread.  A column is kColX cells of x and every y line (the window axis).  Lane
// (lx, g) holds cell lx of the column for the W rows of the window (row r in register
// r mod W, as in 3D); the four lane groups g take different visits of one run (the visits
// with the same first y tap, which all start at the window's first row) and their sums for
// a row are added by two shuffles, in a fixed order, when the row leaves the window.  Staged
// per visit: psi_x in a zero-padded row (as in 3D), psi_y rotated so that register k reads
// its tap at index k and doubled for packed FMAs, c_q and the first y tap.
template <int W, int NS>
struct alignas(16) ColStage2 {
  static constexpr int PY = ((2 * W + 7) / 8) * 8 + 4;   // psi_y rotated, each value twice, padding
  static constexpr int PX = ((W + 15 + 7) / 8) * 8 + 4;  // psi_x at [8, 8 + W)
  float py[NS][PY];
  float px[NS][PX];
  int4 hd[NS];  // byte offset of px[j][8 - ox]; 0; c_q (two floats)
  int sz[NS];   // first y tap
};

template <int W, int NS>
__global__ void __launch_bounds__(kColThreads) k_spread_col2(ColArgs a) {
  using S = ColStage2<W, NS>;
  static_assert(W <= 16 && W % 2 == 0, "rows 0..15 of the window, psi_y read in pairs of taps");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  S* st = reinterpret_cast<S*>(smem_raw) + warp;
  const int lx = lane & 7, g = lane >> 3;
  const int lx4 = 4 * lx;
  const int nfx = a.nf[0], nfy = a.nf[1];
  const unsigned st_off = (unsigned)(reinterpret_cast<unsigned char*>(st) - smem_raw);
  for (int i = lane; i < NS * S::PX; i += 32) (&st->px[0][0])[i] = 0.f;
  __syncwarp();
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(a.counter, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= a.nunits) break;
    const ColUnit U = a.units[u];
    const int x = U.col * kColX + lx;
    const int zpart_hi = U.z1 - U.phi;
    float2 acc[W];
#pragma unroll
    for (int k = 0; k < W; ++k) acc[k] = make_float2(0.f, 0.f);
    int zb = U.z0;
    // row zb leaves the window: the four groups' sums added ((g0 + g1) + (g2 + g3)), written by
    // group 0 (direct, or to a partial slot when other units touch the row)
    auto flush = [&]() {
      float2 v = make_float2(0.f, 0.f);
      switch (zb % W) {
#define DDI_TAKE(R)                          \
  case R:                                    \
    if constexpr (R < W) {                   \
      v = acc[R];                            \
      acc[R] = make_float2(0.f, 0.f);        \
    }                                        \
    break;
        DDI_COL_CASES(DDI_TAKE)
#undef DDI_TAKE
      }
      v.x += __shfl_xor_sync(0xffffffffu, v.x, 8);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, 8);
      v.x += __shfl_xor_sync(0xffffffffu, v.x, 16);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, 16);
      if (g == 0) {
        const int r = zb - U.z0;
        if (r < U.plo || zb >= zpart_hi) {
          const int k = r < U.plo ? r : U.plo + (zb - zpart_hi);
          a.partial[(size_t)__ldg(a.unit_slots + U.slot0 + k) * kColX + lx] = v;
        } else {
          __stcs(a.fine + (long long)(zb >= nfy ? zb - nfy : zb) * nfx + x, v);
        }
      }
      ++zb;
    };
    for (int kb = U.lo; kb < U.hi; kb += NS) {
      const int cnt = min(NS, U.hi - kb);
      bool run_start = false;
      if (lane < cnt) {
        const int2 v = a.visits[kb + lane];
        run_start = (v.y >> 12) & 1;
        const float* ps = a.psi + (size_t)v.x * 3 * W;
        {
          float t[W];
          load_taps<float, W>(ps, t);
#pragma unroll
          for (int k = 0; k < W; ++k) st->px[lane][8 + k] = t[k];
        }
        const int sy = v.y >> 13;
        {
          float t[W];
          load_taps<float, W>(ps + W, t);
          float2* pyr = reinterpret_cast<float2*>(st->py[lane]);
          const int rot = sy % W;  // tap dy feeds row s + dy, held in register (s + dy) mod W
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const int q = rot + k < W ? rot + k : rot + k - W;
            pyr[q] = make_float2(t[k], t[k]);
          }
        }
        const float2 cq = __ldg(a.c + v.x);
        const int ox = (v.y & 63) - 16;
        const unsigned pxo = st_off + (unsigned)(offsetof(S, px) + (lane * S::PX + 8 - ox) * sizeof(float));
        st->hd[lane] = make_int4((int)pxo, 0, __float_as_int(cq.x), __float_as_int(cq.y));
        st->sz[lane] = sy;
      }
      // runs of one first y tap (bit j set where staged visit j starts one; visit 0 always
      // starts the batch's first run)
      unsigned starts = __ballot_sync(0xffffffffu, run_start) | 1u;
      __syncwarp();
      while (starts) {
        const int j0 = __ffs(starts) - 1;
        starts &= starts - 1;
        const int j1 = starts ? __ffs(starts) - 1 : cnt;
        const int sr = st->sz[j0];
        while (zb < sr) flush();
        for (int j = j0 + g; j < j1; j += 4) {
          const int4 h = st->hd[j];
          const float wx = *reinterpret_cast<const float*>(smem_raw + h.x + lx4);
          const float2 cw = make_float2(wx * __int_as_float(h.z), wx * __int_as_float(h.w));
          const float4* p4 = reinterpret_cast<const float4*>(st->py[j]);
#pragma unroll
          for (int k = 0; k < W / 2; ++k) {
            const float4 q = p4[k];
            acc[2 * k] = __ffma2_rn(cw, make_float2(q.x, q.y), acc[2 * k]);
            acc[2 * k + 1] = __ffma2_rn(cw, make_float2(q.z, q.w), acc[2 * k + 1]);
          }
        }
      }
      __syncwarp();
    }
    while (zb < U.z1) flush();
  }
}

// 2D rows that several column units touch: eight lanes per entry (one per cell), the entry's
// partial slots summed in slot order (deterministic), eight loads in flight at a time.
__global__ void __launch_bounds__(256)
    k_reduce_col2(const ColRed* __restrict__ red, int nred, const float2* __restrict__ partial,
                  float2* __restrict__ fine, int nfx) {
  const int e = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 3);
  if (e >= nred) return;
  const int lx = threadIdx.x & 7;
  const int4 r = __ldg(reinterpret_cast<const int4*>(red) + e);  // col, row, s0, ns
  const float2* src = partial + (size_t)r.z * kColX + lx;
  float2 sum = make_float2(0.f, 0.f);
  int k = 0;
  for (; k + 8 <= r.w; k += 8) {
    float2 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcs(src + (size_t)(k + q) * kColX);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sum.x += v[q].x;
      sum.y += v[q].y;
    }
  }
  for (; k < r.w; ++k) {
    const float2 v = __ldcs(src + (size_t)k * kColX);
    sum.x += v.x;
    sum.y += v.y;
  }
  fine[(long long)r.y * nfx + r.x * kColX + lx] = sum;
}

// the column spread kernel of a plan's dimension, and its per-CTA shared memory
template <int W, int NS, bool COMP, int DIM>
struct ColKernel {
  static void (*fn())(ColArgs) { return k_spread_col<W, NS, COMP>; }
  static constexpr size_t smem = sizeof(ColStage<W, NS>) * (kColThreads / 32);
};
template <int W, int NS>
struct ColKernel<W, NS, false, 2> {
  static void (*fn())(ColArgs) { return k_spread_col2<W, NS>; }
  static constexpr size_t smem = sizeof(ColStage2<W, NS>) * (kColThreads / 32);
};

template <int W, int NS, bool COMP, int DIM>
int configure_spread_col(Plan& p) {
  const size_t smem = ColKernel<W, NS, COMP, DIM>::smem;
  auto kern = ColKernel<W, NS, COMP, DIM>::fn();
  {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    DDI_CUDA(cudaFuncGetAttributes(&fa, kern));
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
      DDI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int per_sm = 0;
  DDI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kColThreads, smem));
  int sms = 0;
  DDI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device));
  p.spread_smem = smem;
  p.spread_blocks = std::max(1, std::min(per_sm * sms, (p.ncunits + kColThreads / 32 - 1) / (kColThreads / 32)));
  return DDI_OK;
}

template <int W, int NS, bool COMP, int DIM>
int launch_spread_col(Plan& p, cudaStream_t s) {
  ColArgs a;
  for (int d = 0; d < 3; ++d) a.nf[d] = p.nf[d];
  a.ncx = p.nf[0] / kColX;
  a.units = p.d_cunits;
  a.nunits = p.ncunits;
  a.counter = p.d_counter;
  a.visits = p.d_cvis;
  a.c = static_cast<const float2*>(p.d_c);
  a.psi = static_cast<const float*>(p.d_psi);
  a.fine = static_cast<float2*>(p.d_fine);
  a.partial = static_cast<float2*>(p.d_cpart);
  a.unit_slots = p.d_cslots;
  DDI_CUDA(cudaMemsetAsync(p.d_counter, 0, sizeof(int), s));
  ColKernel<W, NS, COMP, DIM>::fn()<<<p.spread_blocks, kColThreads, p.spread_smem, s>>>(a);
  DDI_LAUNCH_CHECK();
  p.mark("spread", s);
  if (p.ncred > 0) {
    if (DIM == 3)
      k_reduce_col<<<(unsigned)((p.ncred + 7) / 8), 256, 0, s>>>(
          p.d_cred, p.ncred, static_cast<const float2*>(p.d_cpart), static_cast<float2*>(p.d_fine), p.nf[0], p.nf[1],
          a.ncx);
    else
      k_reduce_col2<<<(unsigned)((p.ncred + 31) / 32), 256, 0, s>>>(
          p.d_cred, p.ncred, static_cast<const float2*>(p.d_cpart), static_cast<float2*>(p.d_fine), p.nf[0]);
    DDI_LAUNCH_CHECK();
    p.mark("spread_reduce", s);
  }
  return DDI_OK;
}

template <int W>
int spread_col_ns(Plan& p, cudaStream_t s, bool configure) {
  if (p.dim == 2)  // 2D columns carry no compensated variant (such plans take the tile spread)
    return configure ? configure_spread_col<W, 32, false, 2>(p) : launch_spread_col<W, 32, false, 2>(p, s);
  if (p.col_comp) return configure ? configure_spread_col<W, 32, true, 3>(p) : launch_spread_col<W, 32, true, 3>(p, s);
  return configure ? configure_spread_col<W, 32, false, 3>(p) : launch_spread_col<W, 32, false, 3>(p, s);
}

int spread_col_w(Plan& p, cudaStream_t s, bool configure) {
  switch (p.w) {
    case 6: return spread_col_ns<6>(p, s, configure);
    case 8: return spread_col_ns<8>(p, s, configure);
  }
  set_error("column spread: kernel width %d not built", p.w);
  return DDI_ERR_ARG;
}

// ---- launch helpers ----------------------------------------------------------------------------
template <typename T, int W, int DIM>
int launch_interp(Plan& p, cudaStream_t s) {
  const long long cnt = p.Mh;
  constexpr int XL = W <= 8 ? 8 : 16;
  if (cnt == 0) return DDI_OK;
  k_interp<T, W, DIM><<<(unsigned)((cnt * XL + 255) / 256), 256, 0, s>>>(
      static_cast<const cx_t<T>*>(p.d_fine), static_cast<const ushort4*>(p.d_l0), static_cast<const T*>(p.d_psi),
      static_cast<const T*>(p.d_scale), static_cast<cx_t<T>*>(p.d_c), cnt, dims_of(p));
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
  a.c = p.d_c;
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
    for (int s0 = 0; s0 < p.nsplit; s0 += 65535) {
      const dim3 grid((unsigned)((p.tile[0] * p.tile[1] + 255) / 256), (unsigned)std::min(65535, p.nsplit - s0));
      k_reduce<T, DIM><<<grid, 256, 0, s>>>(p.d_split, static_cast<const cx_t<T>*>(p.d_partial),
                                            static_cast<cx_t<T>*>(p.d_fine), dims_of(p), p.tile[0], p.tile[1],
                                            p.tile[2], p.ntile[0], p.ntile[1], p.ntile[2], s0);
      DDI_LAUNCH_CHECK();
    }
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
DDI_WIDTH_SWITCH(launch_spread)
DDI_WIDTH_SWITCH(configure_spread)

}  // namespace

int configure_kernels(Plan& p) {
  if (p.spread_kind == DDI_SPREAD_COLUMNS) return spread_col_w(p, nullptr, /*configure=*/true);
  if (p.prec == DDI_FP64)
    return p.dim == 3 ? configure_spread_w<double, 3>(p, nullptr) : configure_spread_w<double, 2>(p, nullptr);
  return p.dim == 3 ? configure_spread_w<float, 3>(p, nullptr) : configure_spread_w<float, 2>(p, nullptr);
}

// Device time of the spread (and its partial-plane reduction) for the plan's current
// tile: the best of `reps` timed launches after one untimed one, on zeroed node values
// (the cost depends on the node set and the tile, not on the values).
int time_spread(Plan& p, cudaStream_t s, int reps, float* ms) {
  DDI_CUDA(cudaMemsetAsync(p.d_c, 0, p.cx_size() * (size_t)p.Mh, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    set_error("time_spread: %s", cudaGetErrorString(cudaGetLastError()));
    return DDI_ERR_CUDA;
  }
  auto once = [&]() {
    if (p.spread_kind == DDI_SPREAD_COLUMNS) return spread_col_w(p, s, false);
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
int run_type1(Plan& p, T* phi, cudaStream_t s, bool acc = false) {
  if (p.spread_kind == DDI_SPREAD_COLUMNS) {
    DDI_TRY(spread_col_w(p, s, false));
  } else {
    DDI_TRY((p.dim == 3 ? launch_spread_w<T, 3>(p, s) : launch_spread_w<T, 2>(p, s)));
  }
  return nufft_inverse_fft<T>(p, phi, s, acc);
}

template <typename T>
int run_type1_from_c(Plan& p, T* phi, cudaStream_t s) {
  return run_type1<T>(p, phi, s);
}

template <typename T>
int run_ddi(Plan& p, const T* rho, T* phi, cudaStream_t s) {
  DDI_TRY(run_type2<T>(p, rho, s));
  if (!p.split()) return run_type1<T>(p, phi, s);
  // split plans (Eq. 3.9): the ball's node values are in d_c, so the fine grid is free for
  // the smooth part I_1 until the spread; I_1 reads rho before it writes phi (which may
  // alias rho), and the ball's part I_2 is added to it
  DDI_TRY(split_smooth_part<T>(p, rho, phi, s));
  return run_type1<T>(p, phi, s, /*acc=*/true);
}

template int run_type2<float>(Plan&, const float*, cudaStream_t);
template int run_type2<double>(Plan&, const double*, cudaStream_t);
template int run_type1_from_c<float>(Plan&, float*, cudaStream_t);
template int run_type1_from_c<double>(Plan&, double*, cudaStream_t);
template int run_ddi<float>(Plan&, const float*, float*, cudaStream_t);
template int run_ddi<double>(Plan&, const double*, double*, cudaStream_t);

}  // namespace ddi

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
// with deconvolution by its Fourier transform psihat(2 pi j'/nf).
//
// Kernels (one launch each):
//   fft_nufft.cu forward passes x (fused with the pad and deconvolution), y, z, pruned
//                to the padded block
//   k_interp     f_q = sum over the w^d taps of psi * F, times 2 h^d W_q (one thread per node)
//   k_spread_planes  owner-computes spread: a CTA owns a fine-grid tile and its list of
//                the nodes whose taps reach it; warps own z-planes, so no atomics; the
//                tile is written once; long lists are split into partial tiles
//   k_reduce     sums the partial tiles of split tiles
//   fft_nufft.cu inverse passes z, y, x (pruned to the cropped block, the last fused
//                with crop, deconvolution and real part)
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <numeric>

#include "common.cuh"

namespace ddi {

// ---- error reporting -----------------------------------------------------------------
namespace {
thread_local std::string g_err;
}
void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
const char* last_error() { return g_err.c_str(); }

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename T> struct Pos4 { T x, y, z, w; };

// FP32: the hardware exponential (relative error a few ulp near the kernel centre, where
// psi is O(1); larger only where psi < 1e-6) with an IEEE square root
__device__ __forceinline__ float es_exp(float v) { return __expf(v); }
__device__ __forceinline__ double es_exp(double v) { return exp(v); }
__device__ __forceinline__ float es_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double es_sqrt(double v) { return sqrt(v); }

// psi at the W taps of one axis: x_a = a - W/2 - f, f = s - l0 - W/2 in (-1, 0].
template <typename T, int W>
__device__ __forceinline__ void es_taps(T f, T beta, T* out) {
  const T inv_hw = (T)2 / (T)W;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    const T z = ((T)a - (T)(W / 2) - f) * inv_hw;
    const T zz = z * z;
    out[a] = zz < (T)1 ? es_exp(beta * (es_sqrt((T)1 - zz) - (T)1)) : (T)0;
  }
}

struct GridDims {
  int n[3];
  int nf[3];
};

// i in [0, 2 nf) -> i mod nf
__device__ __forceinline__ int wrap1(int i, int nf) { return i >= nf ? i - nf : i; }
// i in (-nf, 2 nf) -> i mod nf
__device__ __forceinline__ int wrap2(int i, int nf) { return i < 0 ? i + nf : (i >= nf ? i - nf : i); }

// ---- interpolation (type 2) -----------------------------------------------------------------
template <typename T, int W, int DIM>
__global__ void __launch_bounds__(kThreads)
    k_interp(const cx_t<T>* __restrict__ fine, const ushort4* __restrict__ l0,
             const Pos4<T>* __restrict__ pos, cx_t<T>* __restrict__ out, long long count,
             GridDims g, T beta) {
  using C = cx_t<T>;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const ushort4 s = l0[i];
  const Pos4<T> p = pos[i];
  T kx[W], ky[W];
  es_taps<T, W>(p.x, beta, kx);
  es_taps<T, W>(p.y, beta, ky);
  T ar = 0, ai = 0;
  if (DIM == 3) {
    const T inv_hw = (T)2 / (T)W;
#pragma unroll 1
    for (int az = 0; az < W; ++az) {
      // z weight computed on the fly so that no register array is indexed by az
      const T z = ((T)az - (T)(W / 2) - p.z) * inv_hw;
      const T wz = z * z < (T)1 ? es_exp(beta * (es_sqrt((T)1 - z * z) - (T)1)) : (T)0;
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
  out[i] = cmk<C>(p.w * ar, p.w * ai);
}

// ---- spreading (type 1) ------------------------------------------------------------------------
struct SpreadArgs {
  GridDims g;
  int tile[3];
  int ntile[3];
  const SpreadItem* items;
  const int* vlist;  // per-tile visit lists: nodes whose taps reach the tile, by (oz, oy, ox)
  const ushort4* l0;
  const void* pos;
  const void* c;
  void* fine;
  void* partial;
};

// Start of a footprint relative to a tile origin: l0 - T0 wrapped into [-(w-1), nf-(w-1)),
// so that footprints reaching the tile from below (through the periodic wrap) are negative.
__host__ __device__ inline int rel_start(int l0, int T0, int nf, int w) {
  int o = l0 - T0;
  if (o < 0) o += nf;
  if (o > nf - w) o -= nf;
  return o;
}
// Row stride (cells) of the plane-owned accumulator.  A half-warp touches two 8-cell row
// segments; they must fall in different halves of the 128-byte bank window.  Rows of a
// multiple of 16 cells are unpadded and swizzled (x ^ 8 on odd rows); other widths are
// padded to a stride = 8 (mod 16).
__host__ __device__ inline bool spread_swizzle(int TX) { return TX % 16 == 0; }
// first fine cell of tile t along an axis: t T - T/2 (mod nf); unshifted with one tile
__host__ __device__ inline int tile_origin(int t, int T, int ntile, int nf) {
  if (ntile == 1) return 0;
  int o = t * T - T / 2;
  return o < 0 ? o + nf : o;
}
__host__ __device__ inline int spread_row_stride(int TX) {
  return spread_swizzle(TX) ? TX : TX + ((8 - TX % 16) + 16) % 16;
}
__device__ __forceinline__ int spread_cell(int y, int x, int RS, bool swz) {
  return y * RS + (swz ? (x ^ ((y & 1) << 3)) : x);
}

constexpr int kStageS = 64;  // nodes staged per round in k_spread_planes

// Plane-owned spread (no atomics).  A CTA owns a fine-grid tile; its visit list holds
// exactly the nodes whose w^d taps reach the tile, sorted by relative start
// (oz, oy, ox).  After staging a round of nodes (kernel values, c psi_z, starts), warp
// `p mod 8` owns z-plane p of the tile: it binary-searches the staged nodes whose z taps
// cover p, and its lanes (x fastest, then y rows) add c psi_z psi_y psi_x into the
// plane's cells with plain shared-memory read-modify-writes: no other warp touches the
// plane and a lane never meets the same cell twice in one node.  In 2D the owned unit
// is a y-row.
template <typename T, int W, int DIM>
__global__ void __launch_bounds__(kThreads) k_spread_planes(SpreadArgs a, T beta) {
  using C = cx_t<T>;
  constexpr int XL = W <= 8 ? 8 : 16;   // lanes along x
  constexpr int RL = 32 / XL;           // y rows per warp instruction (3D)
  constexpr int MR = (W + RL - 1) / RL; // row iterations per (node, plane)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = a.tile[0], TY = a.tile[1], TZ = a.tile[2];
  const int RS = spread_row_stride(TX);
  const bool swz = spread_swizzle(TX);
  const int NPL = DIM == 3 ? TZ : TY;          // owned units: z-planes (3D) or y-rows (2D)
  const int PSZ = DIM == 3 ? TY * RS : RS;     // cells per owned unit
  C* acc = reinterpret_cast<C*>(smem_raw);     // [NPL][PSZ]
  C* cz = acc + NPL * PSZ;                     // [kStageS][W]: c psi_z (3D) / c psi_y (2D)
  T* py = reinterpret_cast<T*>(cz + kStageS * W);  // [kStageS][W] (3D only)
  T* px = py + kStageS * W;                    // [kStageS][W]
  int* oo = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(px + kStageS * W) + 15) &
                                   ~static_cast<uintptr_t>(15));  // [kStageS][4]: ox, oy, oz, -

  const SpreadItem it = a.items[blockIdx.x];
  const int tx = it.tile % a.ntile[0];
  const int ty = (it.tile / a.ntile[0]) % a.ntile[1];
  const int tz = it.tile / (a.ntile[0] * a.ntile[1]);
  const int nfx = a.g.nf[0], nfy = a.g.nf[1], nfz = a.g.nf[2];
  // the tile lattice is shifted by half a tile so that k = 0 sits inside a tile
  const int T0x = tile_origin(tx, TX, a.ntile[0], nfx);
  const int T0y = tile_origin(ty, TY, a.ntile[1], nfy);
  const int T0z = tile_origin(tz, TZ, a.ntile[2], nfz);
  const bool wrx = a.ntile[0] == 1, wry = a.ntile[1] == 1, wrz = a.ntile[2] == 1;
  const bool wrp = DIM == 3 ? wrz : wry;       // owned axis wraps inside the tile
  const int nfp = DIM == 3 ? nfz : nfy;

  for (int i = threadIdx.x; i < NPL * PSZ; i += blockDim.x) acc[i] = cmk<C>((T)0, (T)0);

  const Pos4<T>* pos = static_cast<const Pos4<T>*>(a.pos);
  const C* cin = static_cast<const C*>(a.c);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rx = lane % XL, ry = lane / XL;

  for (int v0 = it.vbeg; v0 < it.vend; v0 += kStageS) {
    const int cnt = min(kStageS, it.vend - v0);
    __syncthreads();  // the previous round's readers are done
    constexpr int NAX = DIM == 3 ? 3 : 2;
    for (int j = threadIdx.x; j < NAX * cnt; j += blockDim.x) {
      const int ax = j / cnt, k = j - ax * cnt;
      const int node = a.vlist[v0 + k];
      const Pos4<T> pp = pos[node];
      const ushort4 sl = a.l0[node];
      if (ax == 0) {
        es_taps<T, W>(pp.x, beta, px + k * W);
        oo[k * 4 + 0] = rel_start(sl.x, T0x, nfx, W);
      } else if (DIM == 3 && ax == 1) {
        es_taps<T, W>(pp.y, beta, py + k * W);
        oo[k * 4 + 1] = rel_start(sl.y, T0y, nfy, W);
      } else {
        // the owned axis (z in 3D, y in 2D): store c * psi along it
        T w[W];
        es_taps<T, W>(DIM == 3 ? pp.z : pp.y, beta, w);
        const C cq = cin[node];
#pragma unroll
        for (int q = 0; q < W; ++q) cz[k * W + q] = cmk<C>(cq.x * w[q], cq.y * w[q]);
        const int o = DIM == 3 ? rel_start(sl.z, T0z, nfz, W) : rel_start(sl.y, T0y, nfy, W);
        oo[k * 4 + 2] = o;
        if (DIM == 2) oo[k * 4 + 1] = o;
      }
    }
    __syncthreads();
    for (int p = warp; p < NPL; p += kWarps) {
      // staged nodes whose taps along the owned axis cover unit p: key in [p - w + 1, p]
      int lo = 0, hi = cnt;
      if (!wrp) {
        int l = 0, h = cnt;
        while (l < h) { const int m = (l + h) >> 1; if (oo[m * 4 + 2] < p - W + 1) l = m + 1; else h = m; }
        lo = l;
        h = cnt;
        while (l < h) { const int m = (l + h) >> 1; if (oo[m * 4 + 2] <= p) l = m + 1; else h = m; }
        hi = l;
      }
      C* plane = acc + p * PSZ;
      if (!(wrx || wry || wrp)) {
        // fast path: no periodic wrap inside the tile.  Consecutive nodes with the same
        // (oy, ox) hit the same cells of this plane: they are summed in registers and the
        // plane is updated once per run.
        T ar[MR], ai[MR];
#pragma unroll
        for (int m = 0; m < MR; ++m) ar[m] = ai[m] = (T)0;
        int run_x = INT_MIN, run_y = 0;
        for (int k = lo; k <= hi; ++k) {
          int4 o = make_int4(INT_MIN, 0, 0, 0);
          if (k < hi) o = *reinterpret_cast<const int4*>(oo + k * 4);
          if (o.x != run_x || o.y != run_y) {
            if (run_x != INT_MIN) {
              const int xx = run_x + rx;
              if (rx < W && (unsigned)xx < (unsigned)TX) {
#pragma unroll
                for (int m = 0; m < (DIM == 3 ? MR : 1); ++m) {
                  const int r = DIM == 3 ? ry + RL * m : 0;
                  const int yy = run_y + r;
                  if ((DIM == 3 && (r >= W || (unsigned)yy >= (unsigned)TY)) || (DIM == 2 && ry != 0)) continue;
                  C* cell = plane + (DIM == 3 ? spread_cell(yy, xx, RS, swz) : xx);
                  C cur = *cell;
                  cur.x += ar[m];
                  cur.y += ai[m];
                  *cell = cur;
                }
              }
#pragma unroll
              for (int m = 0; m < MR; ++m) ar[m] = ai[m] = (T)0;
            }
            run_x = o.x;
            run_y = o.y;
          }
          if (k == hi) break;
          const C czv = cz[k * W + (p - o.z)];
          const T wx = rx < W ? px[k * W + rx] : (T)0;
#pragma unroll
          for (int m = 0; m < (DIM == 3 ? MR : 1); ++m) {
            const int r = DIM == 3 ? ry + RL * m : 0;
            const T w = DIM == 3 ? (r < W ? py[k * W + r] : (T)0) * wx : wx;
            ar[m] += czv.x * w;
            ai[m] += czv.y * w;
          }
        }
        continue;
      }
      for (int k = lo; k < hi; ++k) {
        int az = p - oo[k * 4 + 2];
        if (wrp) {
          az = az < 0 ? az + nfp : (az >= nfp ? az - nfp : az);
          if (az >= W) continue;
        }
        const int xx0 = oo[k * 4 + 0] + rx;
        const int xx = wrx && xx0 < 0 ? xx0 + nfx : xx0;
        if (rx >= W || xx < 0 || xx >= TX) continue;
        const C czv = cz[k * W + az];
        const T wx = px[k * W + rx];
        if (DIM == 3) {
          const int oy = oo[k * 4 + 1];
#pragma unroll
          for (int m = 0; m < MR; ++m) {
            const int r = ry + RL * m;
            const int yy0 = oy + r;
            const int yy = wry && yy0 < 0 ? yy0 + nfy : yy0;
            if (r < W && yy >= 0 && yy < TY) {
              const T w = py[k * W + r] * wx;
              C* cell = plane + spread_cell(yy, xx, RS, swz);
              C cur = *cell;
              cur.x += czv.x * w;
              cur.y += czv.y * w;
              *cell = cur;
            }
          }
        } else if (ry == 0) {
          C* cell = plane + xx;
          C cur = *cell;
          cur.x += czv.x * wx;
          cur.y += czv.y * wx;
          *cell = cur;
        }
      }
    }
  }
  __syncthreads();
  const int cells = TX * TY * TZ;
  if (it.slot < 0) {
    C* fine = static_cast<C*>(a.fine);
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
      const int gx = T0x + lx, gy = T0y + ly, gz = T0z + lz;
      const long long off = ((long long)(gz >= nfz ? gz - nfz : gz) * nfy + (gy >= nfy ? gy - nfy : gy)) * nfx +
                            (gx >= nfx ? gx - nfx : gx);
      fine[off] = acc[DIM == 3 ? lz * PSZ + spread_cell(ly, lx, RS, swz) : ly * PSZ + lx];
    }
  } else {
    C* part = static_cast<C*>(a.partial) + (long long)it.slot * cells;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
      part[i] = acc[DIM == 3 ? lz * PSZ + spread_cell(ly, lx, RS, swz) : ly * PSZ + lx];
    }
  }
}

constexpr int kStageA = 128;  // nodes staged per round in k_spread_atomic

// plane stride (in cells) of the padded accumulator: >= TY (TX + 1) and = 8 mod 32
__host__ __device__ inline int atomic_plane_stride(int TX, int TY) {
  const int ps = TY * (TX + 1);
  return ps + (((8 - ps) % 32) + 32) % 32;
}

// Owner-computes spread with shared-memory atomics.  A CTA owns a fine-grid tile and
// accumulates every node whose taps reach it.  The staged nodes are split into one
// contiguous slice per warp; lanes own (z, y) rows of the w^d footprint and the w taps
// of each row.  Nodes are sorted by first tap within each bin, so a run of nodes with
// the same footprint (the k ~ 0 hot spot is made of such runs) accumulates in
// registers (REG) and reaches shared memory once per run; rows outside the tile are
// skipped.  Without REG (large widths) every node goes straight to shared memory.
template <typename T, int W, int DIM, bool REG>
__global__ void __launch_bounds__(kThreads) k_spread_atomic(SpreadArgs a, T beta) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = a.tile[0], TY = a.tile[1], TZ = a.tile[2];
  const int cells = TX * TY * TZ;
  // planar re / im accumulators with padded strides: row stride TX + 1 and a plane
  // stride = 8 (mod 32), so the 32 rows a warp touches fall in 32 different banks
  const int RS = TX + 1;
  const int PS = atomic_plane_stride(TX, TY);
  const int cellsP = TZ * PS;
  T* acc = reinterpret_cast<T*>(smem_raw);                      // re [cellsP], im [cellsP]
  C* cv = reinterpret_cast<C*>(acc + 2 * cellsP);               // [kStageA]
  T* kv = reinterpret_cast<T*>(cv + kStageA);                   // [kStageA][3][W]
  int* lv = reinterpret_cast<int*>(kv + kStageA * 3 * W);      // [kStageA][3]

  const SpreadItem it = a.items[blockIdx.x];
  const int tx = it.tile % a.ntile[0];
  const int ty = (it.tile / a.ntile[0]) % a.ntile[1];
  const int tz = it.tile / (a.ntile[0] * a.ntile[1]);
  const int T0x = tile_origin(tx, TX, a.ntile[0], a.g.nf[0]);
  const int T0y = tile_origin(ty, TY, a.ntile[1], a.g.nf[1]);
  const int T0z = tile_origin(tz, TZ, a.ntile[2], a.g.nf[2]);
  for (int i = threadIdx.x; i < 2 * cellsP; i += blockDim.x) acc[i] = (T)0;
  __syncthreads();

  const Pos4<T>* pos = static_cast<const Pos4<T>*>(a.pos);
  const C* cin = static_cast<const C*>(a.c);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int ROWS = DIM == 3 ? W * W : W;   // (z, y) rows of one footprint
  constexpr int RPL = (ROWS + 31) / 32;        // rows per lane
  const int nfx = a.g.nf[0], nfy = a.g.nf[1], nfz = a.g.nf[2];

  for (int v0 = it.vbeg; v0 < it.vend; v0 += kStageA) {
    const int cnt = min(kStageA, it.vend - v0);
    for (int j = threadIdx.x; j < 3 * cnt; j += blockDim.x) {
      const int ax = j / cnt, k = j - ax * cnt;
      if (DIM == 2 && ax == 2) continue;
      const int node = a.vlist[v0 + k];
      const Pos4<T> pp = pos[node];
      es_taps<T, W>(ax == 0 ? pp.x : (ax == 1 ? pp.y : pp.z), beta, kv + (k * 3 + ax) * W);
      if (ax == 0) {
        cv[k] = cin[node];
        const ushort4 sl = a.l0[node];
        lv[k * 3 + 0] = sl.x;
        lv[k * 3 + 1] = sl.y;
        lv[k * 3 + 2] = sl.z;
      }
    }
    __syncthreads();
    const int per = (cnt + kWarps - 1) / kWarps;
    const int k0 = warp * per, k1 = min(cnt, k0 + per);
    if (REG) {
      T ar[RPL][W], ai[RPL][W];
      int lz[RPL], ly[RPL];
      int run = -1;
#pragma unroll
      for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int q = 0; q < W; ++q) ar[i][q] = ai[i][q] = (T)0;
      for (int k = k0; k <= k1; ++k) {
        const bool same = run >= 0 && k < k1 && lv[k * 3] == lv[run * 3] && lv[k * 3 + 1] == lv[run * 3 + 1] &&
                          lv[k * 3 + 2] == lv[run * 3 + 2];
        if (run >= 0 && !same) {
          // flush the finished run into the tile (rows and taps outside it are dropped)
          const int sx = lv[run * 3];
#pragma unroll
          for (int i = 0; i < RPL; ++i) {
            if (lz[i] < TZ && ly[i] < TY) {
              const int base = lz[i] * PS + ly[i] * RS;
#pragma unroll
              for (int q = 0; q < W; ++q) {
                const int lx = wrap2(sx + q - T0x, nfx);
                if (lx < TX) {
                  atomicAdd(acc + base + lx, ar[i][q]);
                  atomicAdd(acc + cellsP + base + lx, ai[i][q]);
                }
                ar[i][q] = ai[i][q] = (T)0;
              }
            }
          }
          run = -1;
        }
        if (k == k1) break;
        if (run < 0) {
          run = k;
#pragma unroll
          for (int i = 0; i < RPL; ++i) {
            const int r = lane + 32 * i;
            const int az = DIM == 3 ? r / W : 0, ay = DIM == 3 ? r - (r / W) * W : r;
            const bool valid = r < ROWS;
            lz[i] = valid ? (DIM == 3 ? wrap2(lv[k * 3 + 2] + az - T0z, nfz) : 0) : TZ;
            ly[i] = valid ? wrap2(lv[k * 3 + 1] + ay - T0y, nfy) : TY;
          }
        }
        const T* kk = kv + k * 3 * W;
        const C cq = cv[k];
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          if (lz[i] < TZ && ly[i] < TY) {
            const int r = lane + 32 * i;
            const int az = DIM == 3 ? r / W : 0, ay = DIM == 3 ? r - (r / W) * W : r;
            const T wzy = (DIM == 3 ? kk[2 * W + az] : (T)1) * kk[W + ay];
            const T czr = cq.x * wzy, czi = cq.y * wzy;
#pragma unroll
            for (int q = 0; q < W; ++q) {
              ar[i][q] += czr * kk[q];
              ai[i][q] += czi * kk[q];
            }
          }
        }
      }
    } else {
      for (int k = k0; k < k1; ++k) {
        const T* kk = kv + k * 3 * W;
        const C cq = cv[k];
        const int sx = lv[k * 3], sy = lv[k * 3 + 1], sz = lv[k * 3 + 2];
        for (int r = lane; r < ROWS; r += 32) {
          const int az = DIM == 3 ? r / W : 0, ay = DIM == 3 ? r - (r / W) * W : r;
          const int z = DIM == 3 ? wrap2(sz + az - T0z, nfz) : 0;
          const int y = wrap2(sy + ay - T0y, nfy);
          if (z >= TZ || y >= TY) continue;
          const T wzy = (DIM == 3 ? kk[2 * W + az] : (T)1) * kk[W + ay];
          const T czr = cq.x * wzy, czi = cq.y * wzy;
          const int base = z * PS + y * RS;
#pragma unroll
          for (int q = 0; q < W; ++q) {
            const int lx = wrap2(sx + q - T0x, nfx);
            if (lx < TX) {
              atomicAdd(acc + base + lx, czr * kk[q]);
              atomicAdd(acc + cellsP + base + lx, czi * kk[q]);
            }
          }
        }
      }
    }
    __syncthreads();
  }

  if (it.slot < 0) {
    C* fine = static_cast<C*>(a.fine);
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lx = i % TX, ly2 = (i / TX) % TY, lz2 = i / (TX * TY);
      const int gx = T0x + lx, gy = T0y + ly2, gz = T0z + lz2;
      const long long off = ((long long)(gz >= nfz ? gz - nfz : gz) * nfy + (gy >= nfy ? gy - nfy : gy)) * nfx +
                            (gx >= nfx ? gx - nfx : gx);
      const int pi = lz2 * PS + ly2 * RS + lx;
      fine[off] = cmk<C>(acc[pi], acc[cellsP + pi]);
    }
  } else {
    C* part = static_cast<C*>(a.partial) + (long long)it.slot * cells;
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lx = i % TX, ly2 = (i / TX) % TY, lz2 = i / (TX * TY);
      const int pi = lz2 * PS + ly2 * RS + lx;
      part[i] = cmk<C>(acc[pi], acc[cellsP + pi]);
    }
  }
}

// Sums the partial tiles of split tiles; blockIdx.y selects a slice of the tile's cells
// so that the few, large split tiles still spread over the whole GPU.
constexpr int kReduceSlices = 8;
template <typename T>
__global__ void k_reduce(const SplitTile* __restrict__ split, const cx_t<T>* __restrict__ partial,
                         cx_t<T>* __restrict__ fine, GridDims g, int TX, int TY, int TZ, int ntx,
                         int nty) {
  using C = cx_t<T>;
  const SplitTile st = split[blockIdx.x];
  const int cells = TX * TY * TZ;
  const int per = (cells + kReduceSlices - 1) / kReduceSlices;
  const int c0 = blockIdx.y * per, c1 = min(cells, c0 + per);
  const int tx = st.tile % ntx, ty = (st.tile / ntx) % nty, tz = st.tile / (ntx * nty);
  for (int i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    T sr = 0, si = 0;
    for (int k = 0; k < st.nslots; ++k) {
      const C v = partial[(long long)(st.slot0 + k) * cells + i];
      sr += v.x;
      si += v.y;
    }
    const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
    int gx = tile_origin(tx, TX, ntx, g.nf[0]) + lx;
    int gy = tile_origin(ty, TY, nty, g.nf[1]) + ly;
    int gz = tile_origin(tz, TZ, g.nf[2] / TZ, g.nf[2]) + lz;
    gx -= gx >= g.nf[0] ? g.nf[0] : 0;
    gy -= gy >= g.nf[1] ? g.nf[1] : 0;
    gz -= gz >= g.nf[2] ? g.nf[2] : 0;
    const long long off = ((long long)gz * g.nf[1] + gy) * g.nf[0] + gx;
    fine[off] = cmk<C>(sr, si);
  }
}

GridDims dims_of(const Plan& p) {
  GridDims g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = p.n[d];
    g.nf[d] = p.nf[d];
  }
  return g;
}


template <typename T, int W, int DIM>
int launch_interp(const Plan& p, cudaStream_t s) {
  const long long cnt = p.Mh;
  k_interp<T, W, DIM><<<(unsigned)((cnt + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      static_cast<const cx_t<T>*>(p.d_fine), static_cast<const ushort4*>(p.d_l0),
      static_cast<const Pos4<T>*>(p.d_pos), static_cast<cx_t<T>*>(p.d_c), cnt, dims_of(p), (T)p.beta);
  DDI_LAUNCH_CHECK();
  return DDI_OK;
}

size_t spread_smem(const Plan& p) {
  const size_t rs = p.real_size(), cs = p.cx_size();
  if (p.spread_method == 2) {
    const size_t cellsP = (size_t)p.tile[2] * atomic_plane_stride(p.tile[0], p.tile[1]);
    return cellsP * cs + kStageA * cs + (size_t)kStageA * 3 * p.w * rs + kStageA * 3 * sizeof(int);
  }
  const size_t rsx = spread_row_stride(p.tile[0]);
  const size_t cells = p.dim == 3 ? (size_t)p.tile[2] * p.tile[1] * rsx : (size_t)p.tile[1] * rsx;
  return cells * cs + (size_t)kStageS * p.w * cs + 2 * (size_t)kStageS * p.w * rs + kStageS * 4 * sizeof(int) + 16;
}

template <typename T, int W, int DIM>
int launch_spread(const Plan& p, cudaStream_t s) {
  SpreadArgs a;
  a.g = dims_of(p);
  for (int d = 0; d < 3; ++d) {
    a.tile[d] = p.tile[d];
    a.ntile[d] = p.ntile[d];
  }
  a.items = p.d_items;
  a.vlist = p.d_vlist;
  a.l0 = static_cast<const ushort4*>(p.d_l0);
  a.pos = p.d_pos;
  a.c = p.d_c;
  a.fine = p.d_fine;
  a.partial = p.d_partial;
  const size_t smem = spread_smem(p);
  auto kern = p.spread_method == 2
                  ? (W <= 8 ? k_spread_atomic<T, W, DIM, true> : k_spread_atomic<T, W, DIM, false>)
                  : k_spread_planes<T, W, DIM>;
  if (smem > 48 * 1024) {
    DDI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  kern<<<p.nitems, kThreads, smem, s>>>(a, (T)p.beta);
  DDI_LAUNCH_CHECK();
  const_cast<Plan&>(p).mark("spread", s);
  if (p.nsplit > 0) {
    k_reduce<T><<<dim3(p.nsplit, kReduceSlices), kThreads, 0, s>>>(p.d_split, static_cast<const cx_t<T>*>(p.d_partial),
                                              static_cast<cx_t<T>*>(p.d_fine), dims_of(p), p.tile[0],
                                              p.tile[1], p.tile[2], p.ntile[0], p.ntile[1]);
    DDI_LAUNCH_CHECK();
    const_cast<Plan&>(p).mark("spread_reduce", s);
  }
  return DDI_OK;
}

template <typename T, int DIM>
int interp_w(const Plan& p, cudaStream_t s) {
  if (sizeof(T) == 4) {
    switch (p.w) {
      case 6: return launch_interp<T, 6, DIM>(p, s);
      case 8: return launch_interp<T, 8, DIM>(p, s);
    }
  } else {
    switch (p.w) {
      case 10: return launch_interp<T, 10, DIM>(p, s);
      case 12: return launch_interp<T, 12, DIM>(p, s);
      case 14: return launch_interp<T, 14, DIM>(p, s);
      case 16: return launch_interp<T, 16, DIM>(p, s);
    }
  }
  set_error("kernel width %d not built for this precision", p.w);
  return DDI_ERR_ARG;
}

template <typename T, int DIM>
int spread_w(const Plan& p, cudaStream_t s) {
  if (sizeof(T) == 4) {
    switch (p.w) {
      case 6: return launch_spread<T, 6, DIM>(p, s);
      case 8: return launch_spread<T, 8, DIM>(p, s);
    }
  } else {
    switch (p.w) {
      case 10: return launch_spread<T, 10, DIM>(p, s);
      case 12: return launch_spread<T, 12, DIM>(p, s);
      case 14: return launch_spread<T, 14, DIM>(p, s);
      case 16: return launch_spread<T, 16, DIM>(p, s);
    }
  }
  set_error("kernel width %d not built for this precision", p.w);
  return DDI_ERR_ARG;
}

}  // namespace

template <typename T>
int run_type2(Plan& p, const T* rho, cudaStream_t s) {
  DDI_TRY(nufft_forward_fft<T>(p, rho, s));
  DDI_TRY((p.dim == 3 ? interp_w<T, 3>(p, s) : interp_w<T, 2>(p, s)));
  p.mark("interp", s);
  return DDI_OK;
}

template <typename T>
int run_type1(Plan& p, T* phi, cudaStream_t s) {
  DDI_TRY(p.dim == 3 ? (spread_w<T, 3>(p, s)) : (spread_w<T, 2>(p, s)));
  return nufft_inverse_fft<T>(p, phi, s);
}

template <typename T>
int run_ddi(Plan& p, const T* rho, T* phi, cudaStream_t s) {
  DDI_TRY(run_type2<T>(p, rho, s));
  return run_type1<T>(p, phi, s);
}

template int run_type2<float>(Plan&, const float*, cudaStream_t);
template int run_type2<double>(Plan&, const double*, cudaStream_t);
template int run_type1<float>(Plan&, float*, cudaStream_t);
template int run_type1<double>(Plan&, double*, cudaStream_t);
template int run_ddi<float>(Plan&, const float*, float*, cudaStream_t);
template int run_ddi<double>(Plan&, const double*, double*, cudaStream_t);

// ---- plan construction ----------------------------------------------------------------------------
namespace {

template <typename T>
void fill_pos(const std::vector<double>& f, const std::vector<double>& sc, std::vector<unsigned char>& out) {
  const size_t n = sc.size();
  out.resize(n * sizeof(Pos4<T>));
  Pos4<T>* o = reinterpret_cast<Pos4<T>*>(out.data());
  for (size_t i = 0; i < n; ++i) {
    o[i].x = (T)f[3 * i];
    o[i].y = (T)f[3 * i + 1];
    o[i].z = (T)f[3 * i + 2];
    o[i].w = (T)sc[i];
  }
}

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

void free_plan(Plan& p) {
  void* ptrs[] = {p.d_l0, p.d_pos, p.d_c, p.d_deconv, p.d_fine, p.d_partial, p.d_bin_start, p.d_vlist, p.d_items,
                  p.d_split, p.d_psi1, p.d_rho, p.d_phi, p.d_work, p.d_work2, p.d_kin, p.d_red, p.d_io_in, p.d_io_out};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (void*& t : p.d_tw)
    if (t) {
      cudaFree(t);
      t = nullptr;
    }
  if (p.h_red) cudaFreeHost(p.h_red);
  if (p.ev_created)
    for (cudaEvent_t& e : p.mark_ev) cudaEventDestroy(e);
}

void choose_tile(Plan& p) {
  // Tiles must be at least w - 1 cells per axis (so a node's taps reach only its own
  // tile and the next one) and divide the fine grid.
  auto pick = [&](int want, int need, int nf) {
    // largest divisor of nf in [need, want], else the smallest divisor >= need
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
      want[0] = 32; want[1] = 32; want[2] = 8;
    } else {
      want[0] = 16; want[1] = 16; want[2] = 16;
    }
  } else {
    want[0] = 64; want[1] = 64; want[2] = 1;
  }
  for (int d = 0; d < 3; ++d) {
    if (p.desc.tile[d] > 0) want[d] = p.desc.tile[d];
    if (d < p.dim && want[d] < need) want[d] = need;
    p.tile[d] = d < p.dim ? pick(want[d], need, p.nf[d]) : 1;
    p.ntile[d] = p.nf[d] / p.tile[d];
  }
}

}  // namespace

int create_plan(Plan& p, const ddi_plan_desc* desc_in, cudaStream_t stream) {
  std::string err;
  DDI_TRY([&]() {
    int s = normalise_desc(desc_in, &p.desc, &err);
    if (s != DDI_OK) set_error("%s", err.c_str());
    return s;
  }());
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
  p.spread_method = d.spread_method == 2 ? 2 : 1;
  build_quadrature(d, &p.quad);
  p.M = p.quad.M;
  choose_tile(p);

  // one node of each (k, -k) pair: the first half of the azimuth
  const int nphi = d.nphi, half = nphi / 2;
  std::vector<int64_t> qs;
  qs.reserve(p.M / 2);
  for (int64_t q = 0; q < p.M; ++q)
    if ((q % nphi) < half) qs.push_back(q);
  p.Mh = (int64_t)qs.size();
  const int dim = d.dim;
  std::vector<int> bin(p.Mh);
  std::vector<unsigned short> l0w(3 * p.Mh, 0);
  std::vector<double> fr(3 * p.Mh, 0.0), sc(p.Mh);
  for (int64_t i = 0; i < p.Mh; ++i) {
    const int64_t q = qs[i];
    int bc[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      const double k = p.quad.k[dim * q + a];
      const int64_t l0 = fine_start(k, p.h[a], p.nf[a], p.w);
      const double scale = (p.h[a] * (double)p.nf[a]) / (2.0 * M_PI);
      const double s = k * scale;
      fr[3 * i + a] = (s - (double)l0) - 0.5 * (double)p.w;
      const int64_t wr = ((l0 % p.nf[a]) + p.nf[a]) % p.nf[a];
      l0w[3 * i + a] = (unsigned short)wr;
      bc[a] = (int)(wr / p.tile[a]);
    }
    bin[i] = (bc[2] * p.ntile[1] + bc[1]) * p.ntile[0] + bc[0];
    sc[i] = 2.0 * p.dv * p.quad.W[q];
  }
  p.nbins = p.ntile[0] * p.ntile[1] * p.ntile[2];
  std::vector<int64_t> perm(p.Mh);
  std::iota(perm.begin(), perm.end(), 0);
  // sort by bin, then by first tap so that nodes with one footprint are consecutive
  std::vector<int64_t> key(p.Mh);
  for (int64_t i = 0; i < p.Mh; ++i)
    key[i] = ((int64_t)l0w[3 * i + 2] * p.nf[1] + l0w[3 * i + 1]) * p.nf[0] + l0w[3 * i];
  std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) {
    return bin[a] != bin[b] ? bin[a] < bin[b] : key[a] < key[b];
  });
  std::vector<int> bin_start(p.nbins + 1, 0);
  for (int64_t i = 0; i < p.Mh; ++i) bin_start[bin[i] + 1]++;
  for (int b = 0; b < p.nbins; ++b) bin_start[b + 1] += bin_start[b];
  p.order.resize(p.Mh);
  std::vector<ushort4> l0s(p.Mh);
  std::vector<double> frs(3 * p.Mh), scs(p.Mh);
  for (int64_t i = 0; i < p.Mh; ++i) {
    const int64_t o = perm[i];
    p.order[i] = qs[o];
    l0s[i] = make_ushort4(l0w[3 * o], l0w[3 * o + 1], l0w[3 * o + 2], 0);
    for (int a = 0; a < 3; ++a) frs[3 * i + a] = fr[3 * o + a];
    scs[i] = sc[o];
  }

  // spread work list: per tile, the nodes whose taps reach it, sorted by their start
  // relative to the tile (oz, oy, ox); long lists are cut into items writing partial tiles
  std::vector<std::vector<std::pair<int64_t, int>>> lists(p.nbins);
  {
    for (int64_t i = 0; i < p.Mh; ++i) {
      int ta[3][2], nt[3];
      const int lv[3] = {l0s[i].x, l0s[i].y, l0s[i].z};
      for (int a = 0; a < 3; ++a) {
        const int l = a < dim ? lv[a] : 0;
        const int w = a < dim ? p.w : 1;
        const int sh = p.ntile[a] > 1 ? p.tile[a] / 2 : 0;  // lattice shift (tile_origin)
        const int t0 = ((l + sh) % p.nf[a]) / p.tile[a];
        const int t1 = ((l + w - 1 + sh) % p.nf[a]) / p.tile[a];
        ta[a][0] = t0;
        ta[a][1] = t1;
        nt[a] = t1 != t0 ? 2 : 1;
      }
      for (int cz = 0; cz < nt[2]; ++cz)
        for (int cy = 0; cy < nt[1]; ++cy)
          for (int cx = 0; cx < nt[0]; ++cx) {
            const int bx = ta[0][cx], by = ta[1][cy], bz = ta[2][cz];
            const int t = (bz * p.ntile[1] + by) * p.ntile[0] + bx;
            const int ox = rel_start(l0s[i].x, tile_origin(bx, p.tile[0], p.ntile[0], p.nf[0]), p.nf[0], p.w);
            const int oy = rel_start(l0s[i].y, tile_origin(by, p.tile[1], p.ntile[1], p.nf[1]), p.nf[1], p.w);
            const int oz = dim == 3 ? rel_start(l0s[i].z, tile_origin(bz, p.tile[2], p.ntile[2], p.nf[2]), p.nf[2], p.w)
                                    : 0;
            // major key: the owned axis (z in 3D, y in 2D); starts lie in [-15, 2048)
            const int64_t key = dim == 3 ? (((int64_t)oz + 32) * 4096 + (oy + 32)) * 4096 + (ox + 32)
                                         : ((int64_t)oy + 32) * 4096 + (ox + 32);
            lists[t].push_back(std::make_pair(key, (int)i));
          }
    }
  }
  long long total = 0;
  for (auto& L : lists) {
    std::stable_sort(L.begin(), L.end(),
                     [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) { return a.first < b.first; });
    total += (long long)L.size();
  }
  p.chunk = d.chunk > 0 ? d.chunk : (int)std::max<long long>(512, total / (152LL * 6));
  std::vector<int> vlist;
  vlist.reserve(total);
  std::vector<SpreadItem> items;
  std::vector<SplitTile> split;
  int slot = 0;
  for (int t = 0; t < p.nbins; ++t) {
    const int beg = (int)vlist.size();
    for (auto& e : lists[t]) vlist.push_back(e.second);
    const int v = (int)lists[t].size();
    if (v <= p.chunk) {
      items.push_back(SpreadItem{t, beg, beg + v, -1});
    } else {
      const int nch = (v + p.chunk - 1) / p.chunk;
      split.push_back(SplitTile{t, slot, nch, 0});
      for (int c = 0; c < nch; ++c)
        items.push_back(SpreadItem{t, beg + c * p.chunk, beg + std::min(v, (c + 1) * p.chunk), slot + c});
      slot += nch;
    }
  }
  p.visits = total;
  // heaviest items first so the long ones start early
  std::stable_sort(items.begin(), items.end(),
                   [](const SpreadItem& a, const SpreadItem& b) { return (a.vend - a.vbeg) > (b.vend - b.vbeg); });
  p.nitems = (int)items.size();
  p.nsplit = (int)split.size();
  p.nslots = slot;

  // deconvolution factors 1/psihat(2 pi j'/nf), j' = j - n/2
  std::vector<double> dc;
  for (int a = 0; a < 3; ++a) {
    for (int j = 0; j < p.n[a]; ++j) {
      if (p.n[a] == 1) {
        dc.push_back(1.0);
      } else {
        const double xi = 2.0 * M_PI * (double)(j - p.n[a] / 2) / (double)p.nf[a];
        dc.push_back(1.0 / es_kernel_hat(xi, p.w, p.beta));
      }
    }
  }

  // device allocations
  const size_t rs = p.real_size(), cs = p.cx_size();
  const size_t cells = (size_t)p.tile[0] * p.tile[1] * p.tile[2];
  DDI_TRY(dev_alloc(p, &p.d_l0, sizeof(ushort4) * p.Mh, "node taps"));
  DDI_TRY(dev_alloc(p, &p.d_pos, 4 * rs * p.Mh, "node positions"));
  DDI_TRY(dev_alloc(p, &p.d_c, cs * p.Mh, "node values"));
  DDI_TRY(dev_alloc(p, &p.d_deconv, rs * dc.size(), "deconvolution"));
  DDI_TRY(dev_alloc(p, &p.d_fine, cs * p.fine_points(), "fine grid"));
  DDI_TRY(dev_alloc(p, &p.d_partial, cs * cells * std::max(1, p.nslots), "partial tiles"));
  DDI_TRY(dev_alloc(p, (void**)&p.d_bin_start, sizeof(int) * bin_start.size(), "bins"));
  DDI_TRY(dev_alloc(p, (void**)&p.d_vlist, sizeof(int) * std::max<size_t>(1, vlist.size()), "visit lists"));
  DDI_TRY(dev_alloc(p, (void**)&p.d_items, sizeof(SpreadItem) * items.size(), "work items"));
  DDI_TRY(dev_alloc(p, (void**)&p.d_split, sizeof(SplitTile) * std::max<size_t>(1, split.size()), "split tiles"));
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
    set_error("cudaMallocHost failed");
    return DDI_ERR_OOM;
  }
  DDI_TRY(dev_alloc(p, &p.d_io_in, rs * N, "host io in"));
  DDI_TRY(dev_alloc(p, &p.d_io_out, rs * N, "host io out"));

  std::vector<unsigned char> posb, dcb(rs * dc.size());
  if (p.prec == DDI_FP64) {
    fill_pos<double>(frs, scs, posb);
    memcpy(dcb.data(), dc.data(), rs * dc.size());
  } else {
    fill_pos<float>(frs, scs, posb);
    for (size_t i = 0; i < dc.size(); ++i) {
      float v = (float)dc[i];
      memcpy(dcb.data() + 4 * i, &v, 4);
    }
  }
  DDI_CUDA(cudaMemcpyAsync(p.d_l0, l0s.data(), sizeof(ushort4) * p.Mh, cudaMemcpyHostToDevice, stream));
  DDI_CUDA(cudaMemcpyAsync(p.d_pos, posb.data(), posb.size(), cudaMemcpyHostToDevice, stream));
  DDI_CUDA(cudaMemcpyAsync(p.d_deconv, dcb.data(), dcb.size(), cudaMemcpyHostToDevice, stream));
  DDI_CUDA(cudaMemcpyAsync(p.d_bin_start, bin_start.data(), sizeof(int) * bin_start.size(), cudaMemcpyHostToDevice,
                           stream));
  if (!vlist.empty())
    DDI_CUDA(cudaMemcpyAsync(p.d_vlist, vlist.data(), sizeof(int) * vlist.size(), cudaMemcpyHostToDevice, stream));
  DDI_CUDA(cudaMemcpyAsync(p.d_items, items.data(), sizeof(SpreadItem) * items.size(), cudaMemcpyHostToDevice,
                           stream));
  if (!split.empty())
    DDI_CUDA(cudaMemcpyAsync(p.d_split, split.data(), sizeof(SplitTile) * split.size(), cudaMemcpyHostToDevice,
                             stream));
  for (int a = 0; a < 3; ++a) {
    if (p.nf[a] > 1) DDI_TRY(make_twiddles(p, p.nf[a]));
    if (p.n[a] > 1) DDI_TRY(make_twiddles(p, p.n[a]));
  }
  // the host vectors above die with this frame: finish the uploads first
  DDI_CUDA(cudaStreamSynchronize(stream));
  if (spread_smem(p) > 200 * 1024) {
    set_error("spread tile needs %zu bytes of shared memory; choose a smaller tile", spread_smem(p));
    return DDI_ERR_ARG;
  }
  return DDI_OK;
}

void destroy_plan(Plan& p) { free_plan(p); }

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
    default: return "unknown ddi status";
  }
}

const char* ddi_last_error(void) { return ddi::last_error(); }

int ddi_quadrature_tables(const ddi_plan_desc* desc, int64_t* M, double* k, double* W, int32_t* l0) {
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
}

int ddi_plan_create(ddi_plan* out, const ddi_plan_desc* desc, void* stream) {
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
  int s = ddi::create_plan(h->p, desc, static_cast<cudaStream_t>(stream));
  if (s != DDI_OK) {
    ddi::destroy_plan(h->p);
    delete h;
    return s;
  }
  *out = h;
  return DDI_OK;
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
  const Plan& p = plan->p;
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
  info->spread_items = p.nitems;
  info->spread_split_tiles = p.nsplit;
  info->interp_items = (int)((p.Mh + 255) / 256);
  info->kmax = p.desc.kmax;
  info->nr = p.desc.nr;
  info->ntheta = p.desc.ntheta;
  info->nphi = p.desc.nphi;
  info->device_bytes = p.bytes;
  return DDI_OK;
}

int ddi_plan_node_order(ddi_plan plan, int64_t* q) {
  if (!plan || !q) {
    ddi::set_error("plan and q must not be NULL");
    return DDI_ERR_ARG;
  }
  memcpy(q, plan->p.order.data(), sizeof(int64_t) * plan->p.order.size());
  return DDI_OK;
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
  DDI_TRY(check_plan_ptrs(plan, rho, phi));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan& p = plan->p;
  if (p.prec == DDI_FP64) return ddi::run_ddi<double>(p, static_cast<const double*>(rho), static_cast<double*>(phi), s);
  return ddi::run_ddi<float>(p, static_cast<const float*>(rho), static_cast<float*>(phi), s);
}

int ddi_apply_host(ddi_plan plan, const void* rho_host, void* phi_host, void* stream) {
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
  DDI_CUDA(cudaStreamSynchronize(s));
  return DDI_OK;
}

int ddi_apply_timed(ddi_plan plan, const void* rho, void* phi, void* stream, const char** names, double* ms,
                    int cap, int* count) {
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
}

int ddi_type2(ddi_plan plan, const void* rho, void* c, void* stream) {
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
}

int ddi_type1(ddi_plan plan, const void* c, void* phi, void* stream) {
  DDI_TRY(check_plan_ptrs(plan, c, phi));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan& p = plan->p;
  DDI_CUDA(cudaMemcpyAsync(p.d_c, c, p.cx_size() * p.Mh, cudaMemcpyDeviceToDevice, s));
  if (p.prec == DDI_FP64) return ddi::run_type1<double>(p, static_cast<double*>(phi), s);
  return ddi::run_type1<float>(p, static_cast<float*>(phi), s);
}

}  // extern "C"

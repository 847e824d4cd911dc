// Stockham FFT core shared by the plain axis passes (fft.cu) and the pruned/fused NUFFT
// passes (fft_nufft.cu): in-register radix-16/8/4/2/3 DFTs, the Stockham stage loop over a
// padded shared-memory line, and a CTA-level kernel that moves LPB lines between global
// memory and shared memory through a load/store policy.
#pragma once
#include <cmath>

#include "common.cuh"

namespace ddi {
namespace fftcore {

// cos(2 pi k / 16), k = 0..15: exact mathematical constants rounded from 40 digits.
#define DDI_C1 0.9238795325112867561281831893967882868224
#define DDI_C2 0.7071067811865475244008443621048490392848
#define DDI_C3 0.3826834323650897717284599840303988667613
__host__ __device__ constexpr double cos16(int k) {
  return (k & 15) == 0   ? 1.0
         : (k & 15) == 1 ? DDI_C1
         : (k & 15) == 2 ? DDI_C2
         : (k & 15) == 3 ? DDI_C3
         : (k & 15) == 4 ? 0.0
         : (k & 15) == 5 ? -DDI_C3
         : (k & 15) == 6 ? -DDI_C2
         : (k & 15) == 7 ? -DDI_C1
         : (k & 15) == 8 ? -1.0
         : (k & 15) == 9 ? -DDI_C1
         : (k & 15) == 10 ? -DDI_C2
         : (k & 15) == 11 ? -DDI_C3
         : (k & 15) == 12 ? 0.0
         : (k & 15) == 13 ? DDI_C3
         : (k & 15) == 14 ? DDI_C2
                          : DDI_C1;
}
__host__ __device__ constexpr double sin16(int k) { return cos16(k + 12); }  // sin x = cos(x - pi/2)

// v * k for a constant k known in FP64.  In FP32 the constant is applied as head + tail
// (k_hi = fl(k), k_lo = fl(k - k_hi)): a single rounded constant would scale every butterfly
// that uses it by the same |w|^2 != 1 (e.g. 1 - 5.7e-8 for the pi/8 pair), a bias that
// accumulates over the stages and, in a time-splitting run, drains the mass step after
// step; with the tail only the unbiased rounding of each operation remains.
template <typename T>
__device__ __forceinline__ T mul_const(T v, double k) {
  if constexpr (sizeof(T) == 4) {
    const float hi = (float)k;
    const float lo = (float)(k - (double)hi);
    return fmaf(v, hi, v * lo);
  } else {
    return v * (T)k;
  }
}

template <int R, int DIR, typename C>
__device__ __forceinline__ C tw_const(C x, int k) {
  // x * exp(DIR * 2 pi i k / R) with the trivial factors special-cased
  if (k == 0) return x;
  if (4 * k == R) return DIR < 0 ? cmk<C>(x.y, -x.x) : cmk<C>(-x.y, x.x);
  const int idx = (k * (16 / R)) & 15;
  const double c = cos16(idx);
  const double s = DIR * sin16(idx);
  return cmk<C>(mul_const(x.x, c) - mul_const(x.y, s), mul_const(x.x, s) + mul_const(x.y, c));
}

// In-register R-point DFT (natural order in and out), radix-2 decimation in time.
template <int R, int DIR, typename C>
struct Dft {
  __device__ __forceinline__ static void run(C* v) {
    C e[R / 2], o[R / 2];
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    Dft<R / 2, DIR, C>::run(e);
    Dft<R / 2, DIR, C>::run(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      const C t = tw_const<R, DIR>(o[k], k);
      v[k] = cadd(e[k], t);
      v[k + R / 2] = csub(e[k], t);
    }
  }
};
template <int DIR, typename C>
struct Dft<1, DIR, C> {
  __device__ __forceinline__ static void run(C*) {}
};
template <int DIR, typename C>
struct Dft<3, DIR, C> {
  // X1,2 = a - (b + c)/2 +- i DIR (sqrt(3)/2) (b - c)
  __device__ __forceinline__ static void run(C* v) {
    using T = decltype(C::x);
    const double s3 = 0.8660254037844386467637231707529361834714;
    const C t1 = cadd(v[1], v[2]);
    const C d = csub(v[1], v[2]);
    const C t2 = cmk<C>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
    const C rot = cmk<C>(-(T)DIR * mul_const(d.y, s3), (T)DIR * mul_const(d.x, s3));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, rot);
    v[2] = csub(t2, rot);
  }
};

__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// radix of the stage that follows sub-transform length NS (16, then 8/4/2, then 3)
__host__ __device__ constexpr int pow2_part(int n) { return n & (-n); }
__host__ __device__ constexpr int radix_for(int N, int NS) {
  return pow2_part(N / NS) >= 16 ? 16 : (pow2_part(N / NS) > 1 ? pow2_part(N / NS) : 3);
}
__host__ __device__ constexpr int max_radix(int N) { return pow2_part(N) >= 16 ? 16 : (pow2_part(N) > 3 ? pow2_part(N) : 3); }

template <int N>
struct Shape {
  static constexpr int RM = max_radix(N);      // largest radix
  static constexpr int TPL = N / RM;           // threads per line
  static constexpr int LS = N + N / 16 + 1;    // padded line stride in shared memory
};

// One Stockham stage of radix R with sub-transform length NS; each thread owns
// G = ceil(RM / R) butterflies of its line (the last ones masked when R does not divide RM).
// PRECISE: apply the twiddle table's tails (FP32), for transforms repeated many times on
// the same data (time splitting), where a rounded twiddle's |w| != 1 would accumulate.
// stage_compute reads the stage's inputs from the line, twiddles and transforms them.
template <typename C, int N, int R, int NS, int DIR, bool PRECISE>
__device__ __forceinline__ void stage_compute(const C* line, int t, const C* __restrict__ tw,
                                              C (&v)[(Shape<N>::RM + R - 1) / R][R]) {
  constexpr int RM = Shape<N>::RM;
  constexpr int TPL = Shape<N>::TPL;
  constexpr int G = (RM + R - 1) / R;
  constexpr int NB = N / R;  // butterflies per line
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = t + g * TPL;  // butterfly index in [0, N/R)
    if (RM % R == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[g][r] = line[pidx(j + r * NB)];
      if (NS > 1) {
        const int jm = j % NS;
        constexpr int STRIDE = N / (NS * R);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const int ti = jm * r * STRIDE;
          C w = tw[ti];
          if (DIR > 0) w.y = -w.y;
          if constexpr (PRECISE && sizeof(w.x) == 4) {
            // head + tail twiddle (the table holds N heads, then N tails)
            C wl = tw[N + ti];
            if (DIR > 0) wl.y = -wl.y;
            const C x = v[g][r];
            v[g][r] = cmk<C>(fmaf(x.x, w.x, fmaf(-x.y, w.y, x.x * wl.x - x.y * wl.y)),
                             fmaf(x.x, w.y, fmaf(x.y, w.x, x.x * wl.y + x.y * wl.x)));
          } else {
            v[g][r] = cmul(v[g][r], w);
          }
        }
      }
      Dft<R, DIR, C>::run(v[g]);
    }
  }
}

// a middle stage: shared memory to shared memory (Stockham output order)
template <typename C, int N, int R, int NS, int DIR, bool PRECISE>
__device__ __forceinline__ void stage(C* line, int t, const C* __restrict__ tw) {
  constexpr int RM = Shape<N>::RM;
  constexpr int TPL = Shape<N>::TPL;
  constexpr int G = (RM + R - 1) / R;
  constexpr int NB = N / R;
  C v[G][R];
  stage_compute<C, N, R, NS, DIR, PRECISE>(line, t, tw, v);
  __syncthreads();
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = t + g * TPL;
    if (RM % R == 0 || j < NB) {
      const int jm = j % NS;
      const int idxD = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) line[pidx(idxD + r * NS)] = v[g][r];
    }
  }
  __syncthreads();
}

// sub-transform length before the last stage
__host__ __device__ constexpr int last_ns(int N, int NS = 1) {
  return NS * radix_for(N, NS) >= N ? NS : last_ns(N, NS * radix_for(N, NS));
}

// the middle stages, from sub-transform length NS up to (not including) STOP
template <typename C, int N, int DIR, int NS, int STOP, bool PRECISE>
struct MidStages {
  __device__ __forceinline__ static void run(C* line, int t, const C* tw) {
    constexpr int R = radix_for(N, NS);
    stage<C, N, R, NS, DIR, PRECISE>(line, t, tw);
    MidStages<C, N, DIR, NS * R, STOP, PRECISE>::run(line, t, tw);
  }
};
template <typename C, int N, int DIR, int STOP, bool PRECISE>
struct MidStages<C, N, DIR, STOP, STOP, PRECISE> {
  __device__ __forceinline__ static void run(C*, int, const C*) {}
};

template <int N>
__host__ __device__ constexpr int lines_per_cta_base() {
  return N <= 16 ? 128 : (N <= 128 ? 2048 / N : 4096 / N);
}

struct LineGeom {
  long long nlines;
  long long l1;    // line L -> (L / l1, L % l1)
  long long s_hi;  // offset of (L / l1)
  long long s_lo;  // offset of (L % l1)
  long long se;    // element stride along the line
};

__device__ __forceinline__ long long line_off(const LineGeom& g, long long L) {
  return (L / g.l1) * g.s_hi + (L % g.l1) * g.s_lo;
}

// Generic batched-line FFT: a policy P supplies nlines(), contig() (element index fastest
// in memory), ref(L) (the line's addresses, computed once per line by one thread),
// load(ref, i) / store(ref, i, v) for element i of the line and kPreciseTwiddles.
// The first Stockham stage takes its inputs straight from global memory and the last one
// writes its outputs straight back (both are in natural element order there), so each
// element crosses shared memory once per middle stage plus once between the first stage
// and the next.  Threads are (line b, butterfly t) pairs: lines fastest when lines are
// strided in memory (a warp's accesses then cover adjacent lines), butterflies fastest
// when lines are contiguous.
template <typename T, int N, int LPB, int DIR, typename P>
__global__ void __launch_bounds__(LPB * Shape<N>::TPL)
    k_fft_policy(P pol, const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  using Ref = typename P::Ref;
  constexpr bool PR = P::kPreciseTwiddles;
  constexpr int LS = Shape<N>::LS;
  constexpr int TPL = Shape<N>::TPL;
  constexpr int RM = Shape<N>::RM;
  constexpr int R0 = radix_for(N, 1);
  static_assert(R0 == RM, "the first stage has one butterfly per thread");
  constexpr int NSL = last_ns(N);      // the last stage's sub-transform length
  constexpr int RL = N / NSL;          // and its radix
  constexpr int GL = (RM + RL - 1) / RL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Ref refs[LPB];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const long long L0 = (long long)blockIdx.x * LPB;
  const long long left = pol.nlines() - L0;
  const int nb = left < LPB ? (int)left : LPB;  // lines of this CTA
  if ((int)threadIdx.x < nb) refs[threadIdx.x] = pol.ref(L0 + threadIdx.x);
  __syncthreads();
  const bool contig = pol.contig();
  const int b = contig ? (int)threadIdx.x / TPL : (int)threadIdx.x % LPB;
  const int t = contig ? (int)threadIdx.x % TPL : (int)threadIdx.x / LPB;
  const bool live = b < nb;
  C* line = sm + b * LS;
  // first stage: butterfly t takes elements t + r N/R0 (all loads issued before use)
  C v0[R0];
#pragma unroll
  for (int r = 0; r < R0; ++r) v0[r] = live ? pol.load(refs[b], t + r * (N / R0)) : cmk<C>((T)0, (T)0);
  Dft<R0, DIR, C>::run(v0);
  if constexpr (R0 == N) {
    // a single stage: outputs in natural order
#pragma unroll
    for (int r = 0; r < R0; ++r)
      if (live) pol.store(refs[b], r, v0[r]);
  } else {
#pragma unroll
    for (int r = 0; r < R0; ++r) line[pidx(t * R0 + r)] = v0[r];
    __syncthreads();
    MidStages<C, N, DIR, R0, NSL, PR>::run(line, t, tw);
    // last stage: butterfly j's outputs are elements j + r NSL
    C v[GL][RL];
    stage_compute<C, N, RL, NSL, DIR, PR>(line, t, tw, v);
#pragma unroll
    for (int g = 0; g < GL; ++g) {
      const int j = t + g * TPL;
      if (live && (RM % RL == 0 || j < N / RL)) {
#pragma unroll
        for (int r = 0; r < RL; ++r) pol.store(refs[b], j + r * NSL, v[g][r]);
      }
    }
  }
}

template <typename T, int N>
constexpr int lines_per_cta() {
  // ~35 KB of shared memory per CTA in FP32, the same line count halved in FP64
  return sizeof(T) == 8 ? (lines_per_cta_base<N>() > 1 ? lines_per_cta_base<N>() / 2 : 1)
                        : lines_per_cta_base<N>();
}

template <typename T, int N, int DIR, typename P>
int launch_policy(const P& pol, const void* tw, cudaStream_t s) {
  constexpr int LPB = lines_per_cta<T, N>();
  constexpr int threads = LPB * Shape<N>::TPL;
  const size_t smem = (size_t)LPB * Shape<N>::LS * sizeof(cx_t<T>);
  auto kern = k_fft_policy<T, N, LPB, DIR, P>;
  if (smem > 48 * 1024) {
    DDI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  const long long blocks = (pol.nlines() + LPB - 1) / LPB;
  if (blocks <= 0) return DDI_OK;
  kern<<<(unsigned)blocks, threads, smem, s>>>(pol, static_cast<const cx_t<T>*>(tw));
  DDI_LAUNCH_CHECK();
  return DDI_OK;
}

// FFT lengths built: 2^a (8..2048) and 3 * 2^a (12..1536)
template <typename T, int DIR, typename P>
int dispatch_policy(int n, const P& pol, const void* tw, cudaStream_t s) {
  switch (n) {
    case 8: return launch_policy<T, 8, DIR>(pol, tw, s);
    case 12: return launch_policy<T, 12, DIR>(pol, tw, s);
    case 16: return launch_policy<T, 16, DIR>(pol, tw, s);
    case 24: return launch_policy<T, 24, DIR>(pol, tw, s);
    case 32: return launch_policy<T, 32, DIR>(pol, tw, s);
    case 48: return launch_policy<T, 48, DIR>(pol, tw, s);
    case 64: return launch_policy<T, 64, DIR>(pol, tw, s);
    case 96: return launch_policy<T, 96, DIR>(pol, tw, s);
    case 128: return launch_policy<T, 128, DIR>(pol, tw, s);
    case 192: return launch_policy<T, 192, DIR>(pol, tw, s);
    case 256: return launch_policy<T, 256, DIR>(pol, tw, s);
    case 384: return launch_policy<T, 384, DIR>(pol, tw, s);
    case 512: return launch_policy<T, 512, DIR>(pol, tw, s);
    case 768: return launch_policy<T, 768, DIR>(pol, tw, s);
    case 1024: return launch_policy<T, 1024, DIR>(pol, tw, s);
    case 1536: return launch_policy<T, 1536, DIR>(pol, tw, s);
    case 2048: return launch_policy<T, 2048, DIR>(pol, tw, s);
    default:
      set_error("FFT length %d not supported (2^a or 3 * 2^a, 8..2048)", n);
      return DDI_ERR_ARG;
  }
}

}  // namespace fftcore
}  // namespace ddi

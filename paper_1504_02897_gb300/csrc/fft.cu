// Batched 1-D complex FFTs along one axis of a 3-D grid (the oversampled NUFFT grid and
// the GPE grid), lengths n = 2^a 3^b.  Stockham autosort formulation: each stage reads
// R values with stride n/R, applies the stage twiddles, does an R-point DFT in
// registers (R = 16 while the power-of-two part allows, then 8/4/2, then 3) and writes
// them back in the next stage's order.  A CTA stages
// LPB lines in shared memory (padded against bank conflicts); lines along y and z are
// loaded LPB at a time so that every global access is a contiguous run of LPB values.
// Twiddles come from an FP64-built table rounded once to the working precision.
#include <cmath>

#include "common.cuh"

namespace ddi {
namespace {

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

template <int R, int DIR, typename C>
__device__ __forceinline__ C tw_const(C x, int k) {
  // x * exp(DIR * 2 pi i k / R) with the trivial factors special-cased
  using T = decltype(C::x);
  if (k == 0) return x;
  if (4 * k == R) return DIR < 0 ? cmk<C>(x.y, -x.x) : cmk<C>(-x.y, x.x);
  const int idx = (k * (16 / R)) & 15;
  const T c = (T)cos16(idx);
  const T s = (T)(DIR * sin16(idx));
  return cmk<C>(x.x * c - x.y * s, x.x * s + x.y * c);
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
    const T s3 = (T)0.8660254037844386467637231707529361834714;
    const C t1 = cadd(v[1], v[2]);
    const C d = csub(v[1], v[2]);
    const C t2 = cmk<C>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
    const C rot = cmk<C>(-(T)DIR * s3 * d.y, (T)DIR * s3 * d.x);
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
template <typename C, int N, int R, int NS, int DIR>
__device__ __forceinline__ void stage(C* line, int t, const C* __restrict__ tw) {
  constexpr int RM = Shape<N>::RM;
  constexpr int TPL = Shape<N>::TPL;
  constexpr int G = (RM + R - 1) / R;
  constexpr int NB = N / R;  // butterflies per line
  C v[G][R];
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
          C w = tw[jm * r * STRIDE];
          if (DIR > 0) w.y = -w.y;
          v[g][r] = cmul(v[g][r], w);
        }
      }
      Dft<R, DIR, C>::run(v[g]);
    }
  }
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

template <typename C, int N, int DIR, int NS>
struct Stages {
  __device__ __forceinline__ static void run(C* line, int t, const C* tw) {
    constexpr int R = radix_for(N, NS);
    stage<C, N, R, NS, DIR>(line, t, tw);
    Stages<C, N, DIR, NS * R>::run(line, t, tw);
  }
};
template <typename C, int N, int DIR>
struct Stages<C, N, DIR, N> {
  __device__ __forceinline__ static void run(C*, int, const C*) {}
};

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

template <typename T, int N, int LPB, int DIR>
__global__ void __launch_bounds__(LPB * Shape<N>::TPL)
    k_fft_lines(cx_t<T>* __restrict__ data, LineGeom g, const cx_t<T>* __restrict__ tw) {
  using C = cx_t<T>;
  constexpr int LS = Shape<N>::LS;
  constexpr int TPL = Shape<N>::TPL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const long long L0 = (long long)blockIdx.x * LPB;
  if (g.se == 1) {
    for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x) {
      const int b = idx / N, i = idx % N;
      const long long L = L0 + b;
      if (L < g.nlines) sm[b * LS + pidx(i)] = data[line_off(g, L) + i];
    }
  } else {
    for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x) {
      const int i = idx / LPB, b = idx % LPB;
      const long long L = L0 + b;
      if (L < g.nlines) sm[b * LS + pidx(i)] = data[line_off(g, L) + (long long)i * g.se];
    }
  }
  __syncthreads();
  const int b = threadIdx.x / TPL;
  const int t = threadIdx.x % TPL;
  Stages<C, N, DIR, 1>::run(sm + b * LS, t, tw);
  if (g.se == 1) {
    for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x) {
      const int bb = idx / N, i = idx % N;
      const long long L = L0 + bb;
      if (L < g.nlines) data[line_off(g, L) + i] = sm[bb * LS + pidx(i)];
    }
  } else {
    for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x) {
      const int i = idx / LPB, bb = idx % LPB;
      const long long L = L0 + bb;
      if (L < g.nlines) data[line_off(g, L) + (long long)i * g.se] = sm[bb * LS + pidx(i)];
    }
  }
}

template <typename T, int N>
constexpr int lines_per_cta() {
  // ~35 KB of shared memory per CTA in FP32, the same line count halved in FP64
  constexpr int base = N <= 16 ? 128 : (N <= 128 ? 2048 / N : 4096 / N);
  return sizeof(T) == 8 ? (base > 1 ? base / 2 : 1) : base;
}

template <typename T, int N, int DIR>
int launch_lines(cx_t<T>* data, const LineGeom& g, const void* tw, cudaStream_t s) {
  constexpr int LPB = lines_per_cta<T, N>();
  constexpr int threads = LPB * Shape<N>::TPL;
  const size_t smem = (size_t)LPB * Shape<N>::LS * sizeof(cx_t<T>);
  auto kern = k_fft_lines<T, N, LPB, DIR>;
  if (smem > 48 * 1024) {
    DDI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  const long long blocks = (g.nlines + LPB - 1) / LPB;
  kern<<<(unsigned)blocks, threads, smem, s>>>(data, g, static_cast<const cx_t<T>*>(tw));
  DDI_LAUNCH_CHECK();
  return DDI_OK;
}

template <typename T, int DIR>
int dispatch(int n, cx_t<T>* data, const LineGeom& g, const void* tw, cudaStream_t s) {
  switch (n) {
    case 8: return launch_lines<T, 8, DIR>(data, g, tw, s);
    case 12: return launch_lines<T, 12, DIR>(data, g, tw, s);
    case 24: return launch_lines<T, 24, DIR>(data, g, tw, s);
    case 48: return launch_lines<T, 48, DIR>(data, g, tw, s);
    case 96: return launch_lines<T, 96, DIR>(data, g, tw, s);
    case 192: return launch_lines<T, 192, DIR>(data, g, tw, s);
    case 384: return launch_lines<T, 384, DIR>(data, g, tw, s);
    case 768: return launch_lines<T, 768, DIR>(data, g, tw, s);
    case 1536: return launch_lines<T, 1536, DIR>(data, g, tw, s);
    case 16: return launch_lines<T, 16, DIR>(data, g, tw, s);
    case 32: return launch_lines<T, 32, DIR>(data, g, tw, s);
    case 64: return launch_lines<T, 64, DIR>(data, g, tw, s);
    case 128: return launch_lines<T, 128, DIR>(data, g, tw, s);
    case 256: return launch_lines<T, 256, DIR>(data, g, tw, s);
    case 512: return launch_lines<T, 512, DIR>(data, g, tw, s);
    case 1024: return launch_lines<T, 1024, DIR>(data, g, tw, s);
    case 2048: return launch_lines<T, 2048, DIR>(data, g, tw, s);
    default:
      set_error("FFT length %d not supported (2^a or 3 * 2^a, 8..2048)", n);
      return DDI_ERR_ARG;
  }
}

}  // namespace

int make_twiddles(Plan& p, int n) {
  if (twiddles(p, n)) return DDI_OK;
  int b = 0;
  while (b < 8 && p.tw_n[b] != 0) ++b;
  if (b == 8) {
    set_error("too many distinct FFT lengths in one plan");
    return DDI_ERR_ARG;
  }
  const size_t es = p.cx_size();
  std::vector<unsigned char> host(es * n);
  for (int k = 0; k < n; ++k) {
    // e^{-2 pi i k / n} from FP64 libm, rounded once to the working precision
    const double ang = (-2.0 * M_PI * (double)k) / (double)n;
    const double c = std::cos(ang), sn = std::sin(ang);
    if (p.prec == DDI_FP64) {
      double2 v = make_double2(c, sn);
      memcpy(host.data() + es * k, &v, es);
    } else {
      float2 v = make_float2((float)c, (float)sn);
      memcpy(host.data() + es * k, &v, es);
    }
  }
  void* d = nullptr;
  if (cudaMalloc(&d, es * n) != cudaSuccess) {
    set_error("cudaMalloc of a twiddle table failed");
    return DDI_ERR_OOM;
  }
  p.bytes += es * n;
  DDI_CUDA(cudaMemcpy(d, host.data(), es * n, cudaMemcpyHostToDevice));
  p.d_tw[b] = d;
  p.tw_n[b] = n;
  return DDI_OK;
}

template <typename T>
int fft_axis(const Plan& p, cx_t<T>* data, int nx, int ny, int nz, int axis, int dir, cudaStream_t s) {
  LineGeom g{};
  int n = 1;
  if (axis == 0) {
    n = nx;
    g.nlines = (long long)ny * nz;
    g.l1 = ny;
    g.s_hi = (long long)nx * ny;
    g.s_lo = nx;
    g.se = 1;
  } else if (axis == 1) {
    n = ny;
    g.nlines = (long long)nx * nz;
    g.l1 = nx;
    g.s_hi = (long long)nx * ny;
    g.s_lo = 1;
    g.se = nx;
  } else {
    n = nz;
    g.nlines = (long long)nx * ny;
    g.l1 = nx;
    g.s_hi = nx;
    g.s_lo = 1;
    g.se = (long long)nx * ny;
  }
  if (n == 1) return DDI_OK;
  const void* tw = twiddles(p, n);
  if (!tw) {
    set_error("missing twiddle table for FFT length %d", n);
    return DDI_ERR_ARG;
  }
  return dir < 0 ? dispatch<T, -1>(n, data, g, tw, s) : dispatch<T, +1>(n, data, g, tw, s);
}

template <typename T>
int fft_3d(const Plan& p, cx_t<T>* data, int nx, int ny, int nz, int dir, cudaStream_t s) {
  DDI_TRY(fft_axis<T>(p, data, nx, ny, nz, 0, dir, s));
  DDI_TRY(fft_axis<T>(p, data, nx, ny, nz, 1, dir, s));
  DDI_TRY(fft_axis<T>(p, data, nx, ny, nz, 2, dir, s));
  return DDI_OK;
}

template int fft_axis<float>(const Plan&, float2*, int, int, int, int, int, cudaStream_t);
template int fft_axis<double>(const Plan&, double2*, int, int, int, int, int, cudaStream_t);
template int fft_3d<float>(const Plan&, float2*, int, int, int, int, cudaStream_t);
template int fft_3d<double>(const Plan&, double2*, int, int, int, int, cudaStream_t);

}  // namespace ddi

// Plain batched 1-D FFTs along one axis of a [nz][ny][nx] complex grid (GPE grid and
// tests) and the FP64-built twiddle tables.  The Stockham core is in fft_core.cuh.
#include <cstring>

#include "fft_core.cuh"

namespace ddi {
namespace {
using namespace fftcore;

template <typename T>
struct PlainLines {
  using C = cx_t<T>;
  C* data;
  LineGeom g;
  using Ref = long long;  // offset of the line's first element
  static constexpr bool kPreciseTwiddles = true;  // the GPE's repeated transforms
  __host__ __device__ long long nlines() const { return g.nlines; }
  __device__ bool contig() const { return g.se == 1; }
  __device__ Ref ref(long long L) const { return line_off(g, L); }
  __device__ C load(Ref r, int i) const { return __ldg(data + r + (long long)i * g.se); }
  __device__ void store(Ref r, int i, C v) const { data[r + (long long)i * g.se] = v; }
};

}  // namespace

int make_twiddles(Plan& p, int n) {
  if (twiddles(p, n)) return DDI_OK;
  int b = 0;
  while (b < 8 && p.tw_n[b] != 0) ++b;
  if (b == 8) {
    set_error("too many distinct FFT lengths in one plan");
    return DDI_ERR_ARG;
  }
  // FP64: e^{-2 pi i k / n} from FP64 libm.  FP32: head and tail of each component,
  // [n] heads then [n] tails, so that a stage multiplies by the twiddle to FP64 accuracy:
  // a rounded twiddle has |w| != 1 by up to 6e-8, and the same table in every transform
  // would scale the data's norm by the same amount every time (a steady mass drift in
  // long time-splitting runs)
  const size_t es = p.cx_size();
  const size_t count = p.prec == DDI_FP64 ? (size_t)n : 2 * (size_t)n;
  std::vector<unsigned char> host(es * count);
  for (int k = 0; k < n; ++k) {
    const double ang = (-2.0 * M_PI * (double)k) / (double)n;
    const double c = std::cos(ang), sn = std::sin(ang);
    if (p.prec == DDI_FP64) {
      double2 v = make_double2(c, sn);
      memcpy(host.data() + es * k, &v, es);
    } else {
      const float ch = (float)c, sh = (float)sn;
      float2 hi = make_float2(ch, sh);
      float2 lo = make_float2((float)(c - (double)ch), (float)(sn - (double)sh));
      memcpy(host.data() + es * k, &hi, es);
      memcpy(host.data() + es * (n + (size_t)k), &lo, es);
    }
  }
  void* d = nullptr;
  if (cudaMalloc(&d, es * count) != cudaSuccess) {
    set_error("cudaMalloc of a twiddle table failed");
    return DDI_ERR_OOM;
  }
  p.bytes += es * count;
  DDI_CUDA(cudaMemcpy(d, host.data(), es * count, cudaMemcpyHostToDevice));
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
  PlainLines<T> pol{data, g};
  return dir < 0 ? dispatch_policy<T, -1>(n, pol, tw, s) : dispatch_policy<T, +1>(n, pol, tw, s);
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

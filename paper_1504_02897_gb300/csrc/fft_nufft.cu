// Fine-grid FFTs of the NUFFT with the zero padding and the cropping built in.
//
// The type-2 input occupies the n^d centred positions j' mod nf (j' = -n/2..n/2-1) of the
// 2n-oversampled grid and the type-1 output is read back at the same positions, so:
//   forward  x: only the n^(d-1) rows through the padded block exist; their input is
//               rho / psihat read straight from rho (pad and deconvolution fused);
//            y: only the planes z in the block; elements outside the block read as zero;
//               only the y lines that hold node taps are stored;
//            z: the columns on those y lines; elements outside the block read as zero.
//   inverse  z: the columns on those y lines; only the z in the block are stored;
//            y: only the planes z in the block; elements on the other y lines read as
//               zero (no tap reaches them); only the y in the block are stored;
//            x: only the rows in the block; the x in the block are stored as
//               Re(u) / psihat into phi (crop, deconvolution and real part fused).
// The y lines with taps: one node of each (k, -k) pair is processed, the one with k_y >= 0
// (the first half of the azimuth), so the taps lie on about half of the y lines (the plan
// finds the shortest cyclic range holding all of them).
// The NUFFT passes run once per evaluation and use the twiddles' FP32 heads only (the
// path's error budget is 1e-6); the GPE's repeated transforms use heads and tails.
// Split plans (Eq. 3.9) run the same six passes a second time for the smooth part I_1,
// without the deconvolution and with the symbol p applied as the forward z pass stores.
// Grid positions that are not read are never written in the same evaluation, so no
// zero-fill of the fine grid is needed.  Each CTA reads its own lines before it writes
// them and no other CTA touches them, so the in-place passes may load through the
// read-only data cache.
#include "fft_core.cuh"

namespace ddi {
namespace {
using namespace fftcore;

struct Axis {
  int n;   // grid points
  int nf;  // fine points
  __host__ __device__ bool in_block(int l) const { return l < n / 2 || l >= nf - n / 2; }
  // grid index j (0..n-1) of fine position l in the block
  __host__ __device__ int grid_of(int l) const { return l < n / 2 ? l + n / 2 : l - (nf - n / 2); }
  // fine position of grid index j
  __host__ __device__ int fine_of(int j) const { return j < n / 2 ? j - n / 2 + nf : j - n / 2; }
};

template <typename T>
struct Geo {
  using C = cx_t<T>;
  Axis ax, ay, az;
  // deconvolution factors 1 / psihat, FP64 (x: [0, n0), y: [n0, n0 + n1), z: after), and for
  // FP32 plans the x factors as FP32 head + tail pairs (the FP64 value to ~2^-48)
  const double* dc;
  const float2* dcx2;
  C* fine;
  // the fine-grid y lines that hold node taps: ylo, ylo + 1, .. (mod nf_y), nyr of them; and
  // the x lines (xlo, .., nxr of them; every line except for split plans' ball)
  int ylo, nyr;
  int xlo, nxr;
  int* nonfinite;  // set when the pad pass reads a NaN / Inf
  __device__ long long fidx(int lz, int ly, int lx) const {
    return ((long long)lz * ay.nf + ly) * ax.nf + lx;
  }
  __host__ __device__ bool in_yr(int l) const {
    int d = l - ylo;
    if (d < 0) d += ay.nf;
    return d < nyr;
  }
  __host__ __device__ bool in_xr(int l) const {
    int d = l - xlo;
    if (d < 0) d += ax.nf;
    return d < nxr;
  }
  __host__ __device__ int yr_line(int i) const {
    const int l = ylo + i;
    return l >= ay.nf ? l - ay.nf : l;
  }
};

// forward x with the pad: lines = grid rows (jy, jz)
template <typename T>
struct RowRef {
  long long grid;  // offset of the row in rho / phi
  long long fine;  // offset of the row in the fine grid
  T hi, lo;        // the row's deconvolution factor dy dz (FP64 product): FP64 value, or FP32 head + tail
};

// the row (jy, jz) of a line: offsets and its factor dy dz, formed in FP64
template <typename T>
__device__ __forceinline__ RowRef<T> row_ref(const Geo<T>& g, long long L) {
  const int jy = (int)(L % g.ay.n), jz = (int)(L / g.ay.n);
  const double f = g.dc[g.ax.n + jy] * g.dc[g.ax.n + g.ay.n + jz];
  RowRef<T> r;
  r.grid = L * g.ax.n;
  r.fine = g.fidx(g.az.fine_of(jz), g.ay.fine_of(jy), 0);
  r.hi = (T)f;
  r.lo = sizeof(T) == 4 ? (T)(f - (double)r.hi) : (T)0;
  return r;
}

// v times the deconvolution factor of element jx of row r, rounded once: in FP64 directly;
// in FP32 the factor dx dy dz is formed as a head + tail pair (the exact product error of the
// heads by an FMA plus the cross terms), so only the final product is rounded
template <typename T>
__device__ __forceinline__ T deconv(const Geo<T>& g, const RowRef<T>& r, int jx, T v) {
  if constexpr (sizeof(T) == 8) {
    return v * (g.dc[jx] * r.hi);
  } else {
    const float2 fx = __ldg(g.dcx2 + jx);
    const float ph = fx.x * r.hi;
    const float pe = fmaf(fx.x, r.hi, -ph) + fmaf(fx.x, r.lo, fx.y * r.hi);
    return fmaf(v, ph, v * pe);
  }
}

template <typename T>
struct PadX {
  using C = cx_t<T>;
  using Ref = RowRef<T>;
  static constexpr bool kPreciseTwiddles = false;
  Geo<T> g;
  const T* rho;
  __host__ __device__ long long nlines() const { return (long long)g.ay.n * g.az.n; }
  __device__ bool contig() const { return true; }
  __device__ Ref ref(long long L) const { return row_ref<T>(g, L); }
  __device__ C load(const Ref& r, int i) const {
    if (!g.ax.in_block(i)) return cmk<C>((T)0, (T)0);
    const int jx = g.ax.grid_of(i);
    const T v = __ldg(rho + r.grid + jx);
    if (!isfinite(v) && *(volatile int*)g.nonfinite == 0) atomicOr(g.nonfinite, 1);
    return cmk<C>(deconv<T>(g, r, jx, v), (T)0);
  }
  __device__ void store(const Ref& r, int i, C v) const { g.fine[r.fine + i] = v; }
};

// y lines of the planes z in the block: forward (pruned input; only the y lines that hold
// node taps are stored) or inverse (pruned output; the y lines without taps are zero)
template <typename T, bool FWD>
struct BlockY {
  using C = cx_t<T>;
  static constexpr bool kPreciseTwiddles = false;
  using Ref = long long;  // fine-grid offset of the line's first element
  Geo<T> g;
  __host__ __device__ long long nlines() const { return (long long)g.ax.nf * g.az.n; }
  __device__ bool contig() const { return false; }
  __device__ Ref ref(long long L) const {
    return g.fidx(g.az.fine_of((int)(L / g.ax.nf)), 0, (int)(L % g.ax.nf));
  }
  __device__ C load(Ref r, int i) const {
    if (FWD ? !g.ay.in_block(i) : !g.in_yr(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + r + (long long)i * g.ax.nf);
  }
  __device__ void store(Ref r, int i, C v) const {
    if (FWD ? !g.in_yr(i) : !g.ay.in_block(i)) return;
    g.fine[r + (long long)i * g.ax.nf] = v;
  }
};

// z columns whose y line holds node taps: forward (pruned input) or inverse (pruned output)
template <typename T, bool FWD>
struct AllZ {
  using C = cx_t<T>;
  static constexpr bool kPreciseTwiddles = false;
  using Ref = long long;  // the column's (y, x) offset
  Geo<T> g;
  __host__ __device__ long long nlines() const { return (long long)g.ax.nf * g.nyr; }
  __device__ bool contig() const { return false; }
  __device__ Ref ref(long long L) const {
    return (long long)g.yr_line((int)(L / g.ax.nf)) * g.ax.nf + L % g.ax.nf;
  }
  __device__ C load(Ref r, int i) const {
    if (FWD && !g.az.in_block(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + (long long)i * g.ay.nf * g.ax.nf + r);
  }
  __device__ void store(Ref r, int i, C v) const {
    if (!FWD && !g.az.in_block(i)) return;
    g.fine[(long long)i * g.ay.nf * g.ax.nf + r] = v;
  }
};

// The band of fine-grid lines around k = 0 that holds every tap of a split plan's ball
// nodes: index i = 0..2b of the band is fine position i (i <= b) or nf - (2b + 1 - i).
__host__ __device__ inline int band_line(int i, int b, int nf) { return i <= b ? i : nf - (2 * b + 1 - i); }

// y lines of the planes z in the block, only the x-columns in the band (split plans' ball)
template <typename T, bool FWD>
struct BandY {
  using C = cx_t<T>;
  static constexpr bool kPreciseTwiddles = false;
  using Ref = long long;  // fine-grid offset of the line's first element
  Geo<T> g;
  int bx;
  __host__ __device__ long long nlines() const { return (long long)(2 * bx + 1) * g.az.n; }
  __device__ bool contig() const { return false; }
  __device__ Ref ref(long long L) const {
    const int wx = 2 * bx + 1;
    return g.fidx(g.az.fine_of((int)(L / wx)), 0, band_line((int)(L % wx), bx, g.ax.nf));
  }
  __device__ C load(Ref r, int i) const {
    // inverse: the spread wrote only the band's y lines (the others hold no tap)
    if (FWD ? !g.ay.in_block(i) : !g.in_yr(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + r + (long long)i * g.ax.nf);
  }
  __device__ void store(Ref r, int i, C v) const {
    if (!FWD && !g.ay.in_block(i)) return;
    g.fine[r + (long long)i * g.ax.nf] = v;
  }
};

// z columns in the band of x and y (split plans' ball)
template <typename T, bool FWD>
struct BandZ {
  using C = cx_t<T>;
  static constexpr bool kPreciseTwiddles = false;
  using Ref = long long;  // the column's (y, x) offset
  Geo<T> g;
  int bx, by;
  __host__ __device__ long long nlines() const { return (long long)(2 * bx + 1) * (2 * by + 1); }
  __device__ bool contig() const { return false; }
  __device__ Ref ref(long long L) const {
    const int wx = 2 * bx + 1;
    const int lx = band_line((int)(L % wx), bx, g.ax.nf), ly = band_line((int)(L / wx), by, g.ay.nf);
    return (long long)ly * g.ax.nf + lx;
  }
  __device__ C load(Ref r, int i) const {
    if (FWD && !g.az.in_block(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + (long long)i * g.ay.nf * g.ax.nf + r);
  }
  __device__ void store(Ref r, int i, C v) const {
    if (!FWD && !g.az.in_block(i)) return;
    g.fine[(long long)i * g.ay.nf * g.ax.nf + r] = v;
  }
};

// inverse x with crop, deconvolution and real part: lines = grid rows (jy, jz); ACC adds
// the result to phi instead of storing it
template <typename T, bool ACC>
struct CropX {
  using C = cx_t<T>;
  using Ref = RowRef<T>;
  static constexpr bool kPreciseTwiddles = false;
  Geo<T> g;
  T* phi;
  __host__ __device__ long long nlines() const { return (long long)g.ay.n * g.az.n; }
  __device__ bool contig() const { return true; }
  __device__ Ref ref(long long L) const { return row_ref<T>(g, L); }
  __device__ C load(const Ref& r, int i) const {
    // x lines outside the taps' range were neither written by the spread nor transformed
    if (!g.in_xr(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + r.fine + i);
  }
  __device__ void store(const Ref& r, int i, C v) const {
    if (!g.ax.in_block(i)) return;
    const int jx = g.ax.grid_of(i);
    const T val = deconv<T>(g, r, jx, v.x);
    if (ACC)
      phi[r.grid + jx] += val;
    else
      phi[r.grid + jx] = val;
  }
};

// The smooth symbol of the split algorithm (Eq. 3.9) at the fine grid's modes,
//   p(k) = (1 - e^{-|k|^2/k0^2}) / |k|^2 * (3 (n.k)(m.k) - (n.m) |k|^2),  p(0) = 0,
// times the inverse transform's 1 / (nf0 nf1 nf2).  Mode l of an axis with nf points is the
// wavenumber (2 pi / (nf h)) l~ with l~ = l for l < nf/2, else l - nf.
template <typename T>
struct SmoothSymbol {
  T dk[3];    // 2 pi / (nf_d h_d)
  T n[3], m[3];
  T nm;       // n.m
  T inv_k02;  // 1 / k0^2
  T scale;    // 1 / (nf0 nf1 nf2)
  __host__ __device__ T k_of(int a, int l, int nf) const { return dk[a] * (T)(l < nf / 2 ? l : l - nf); }
  __device__ T operator()(T kx, T ky, T kz) const {
    const T k2 = (kx * kx + ky * ky) + kz * kz;
    const T nk = (n[0] * kx + n[1] * ky) + n[2] * kz;
    const T mk = (m[0] * kx + m[1] * ky) + m[2] * kz;
    const T poly = (T)3 * (nk * mk) - nm * k2;
    T f;
    if (k2 > (T)0) {
      if constexpr (sizeof(T) == 4)
        f = -expm1f(-(k2 * inv_k02)) / k2;
      else
        f = -expm1(-(k2 * inv_k02)) / k2;
    } else {
      f = inv_k02;
    }
    return (f * poly) * scale;
  }
};

// forward z of the split algorithm's smooth part, with the symbol applied as the
// transformed column is stored: lines = columns (ly, lx) of the fine grid
template <typename T>
struct ZRef {
  long long col;  // the column's (y, x) offset
  T kx, ky;       // the column's x and y wavenumbers
};

template <typename T>
struct SmoothZ {
  using C = cx_t<T>;
  using Ref = ZRef<T>;
  static constexpr bool kPreciseTwiddles = false;
  Geo<T> g;
  SmoothSymbol<T> sy;
  __host__ __device__ long long nlines() const { return (long long)g.ax.nf * g.ay.nf; }
  __device__ bool contig() const { return false; }
  __device__ Ref ref(long long L) const {
    const int lx = (int)(L % g.ax.nf), ly = (int)(L / g.ax.nf);
    return Ref{L, sy.k_of(0, lx, g.ax.nf), sy.k_of(1, ly, g.ay.nf)};
  }
  __device__ C load(const Ref& r, int i) const {
    if (!g.az.in_block(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + (long long)i * g.ay.nf * g.ax.nf + r.col);
  }
  __device__ void store(const Ref& r, int i, C v) const {
    g.fine[(long long)i * g.ay.nf * g.ax.nf + r.col] = cscale(v, sy(r.kx, r.ky, sy.k_of(2, i, g.az.nf)));
  }
};

// unit: the split algorithm's smooth part (a full convolution: every y line, no deconvolution)
template <typename T>
Geo<T> geo_of(Plan& p, bool unit = false) {
  Geo<T> g;
  g.ax = Axis{p.n[0], p.nf[0]};
  g.ay = Axis{p.n[1], p.nf[1]};
  g.az = Axis{p.n[2], p.nf[2]};
  g.ylo = unit ? 0 : p.yr[0];
  g.nyr = unit ? p.nf[1] : p.yr[1];
  g.xlo = unit ? 0 : p.xr[0];
  g.nxr = unit ? p.nf[0] : p.xr[1];
  g.nonfinite = p.d_nonfinite;
  g.dc = static_cast<const double*>(unit ? p.d_ones : p.d_deconv);
  g.dcx2 = static_cast<const float2*>(unit ? p.d_ones_x2 : p.d_deconv_x2);
  g.fine = static_cast<cx_t<T>*>(p.d_fine);
  return g;
}

// a policy with the twiddles applied as head + tail (FP32 tables hold both)
template <typename P>
struct Precise : P {
  static constexpr bool kPreciseTwiddles = true;
};

// one pass of the NUFFT's fine-grid transforms, with precise twiddles when the plan asks
template <typename T, int DIR, typename P>
int pass(Plan& p, int n, const P& pol, cudaStream_t s) {
  if (p.precise_nufft) return dispatch_policy<T, DIR>(n, Precise<P>{pol}, twiddles(p, n), s);
  return dispatch_policy<T, DIR>(n, pol, twiddles(p, n), s);
}

}  // namespace

// split plans with a band: the ball's taps lie in the x-band (y pass) and the x/y band (z
// pass), so only those lines are transformed; interpolation reads nothing else
template <typename T>
bool use_band(const Plan& p) {
  return p.dim == 3 && p.band[0] > 0 && p.band[1] > 0;
}

template <typename T>
int nufft_forward_fft(Plan& p, const T* rho, cudaStream_t s) {
  const Geo<T> g = geo_of<T>(p);
  DDI_TRY((pass<T, -1>(p, p.nf[0], PadX<T>{g, rho}, s)));
  p.mark("pad_fft_x", s);
  if (use_band<T>(p)) {
    DDI_TRY((pass<T, -1>(p, p.nf[1], BandY<T, true>{g, p.band[0]}, s)));
    p.mark("band_fft_y_fwd", s);
    DDI_TRY((pass<T, -1>(p, p.nf[2], BandZ<T, true>{g, p.band[0], p.band[1]}, s)));
    p.mark("band_fft_z_fwd", s);
    return DDI_OK;
  }
  DDI_TRY((pass<T, -1>(p, p.nf[1], BlockY<T, true>{g}, s)));
  p.mark("fft_y_fwd", s);
  if (p.dim == 3) {
    DDI_TRY((pass<T, -1>(p, p.nf[2], AllZ<T, true>{g}, s)));
    p.mark("fft_z_fwd", s);
  }
  return DDI_OK;
}

template <typename T>
int nufft_inverse_fft(Plan& p, T* phi, cudaStream_t s, bool acc) {
  const Geo<T> g = geo_of<T>(p);
  if (use_band<T>(p)) {
    // the spread wrote every fine cell, zero off the taps, so the skipped lines are zero
    // before and after their transforms, as the crop expects
    DDI_TRY((pass<T, +1>(p, p.nf[2], BandZ<T, false>{g, p.band[0], p.band[1]}, s)));
    p.mark("band_fft_z_inv", s);
    DDI_TRY((pass<T, +1>(p, p.nf[1], BandY<T, false>{g, p.band[0]}, s)));
    p.mark("band_fft_y_inv", s);
  } else {
    if (p.dim == 3) {
      DDI_TRY((pass<T, +1>(p, p.nf[2], AllZ<T, false>{g}, s)));
      p.mark("fft_z_inv", s);
    }
    DDI_TRY((pass<T, +1>(p, p.nf[1], BlockY<T, false>{g}, s)));
    p.mark("fft_y_inv", s);
  }
  if (acc)
    DDI_TRY((pass<T, +1>(p, p.nf[0], CropX<T, true>{g, phi}, s)));
  else
    DDI_TRY((pass<T, +1>(p, p.nf[0], CropX<T, false>{g, phi}, s)));
  p.mark(acc ? "fft_x_inv_crop_add" : "fft_x_inv_crop", s);
  return DDI_OK;
}

// I_1 of Eq. 3.9: rho zero-padded into the fine grid (the centred block, as for the NUFFT,
// which leaves the circular convolution unchanged), forward x, y, z with p applied as z is
// stored, inverse z, y, x, crop and real part.  The 2x padding makes the circular
// convolution linear up to the kernel's tail beyond one box length.
template <typename T>
int split_smooth_part(Plan& p, const T* rho, T* phi, cudaStream_t s) {
  if (p.dim != 3 || !p.split() || !p.d_ones) {
    set_error("split_smooth_part: not a 3D split plan");
    return DDI_ERR_ARG;
  }
  const Geo<T> g = geo_of<T>(p, /*unit=*/true);
  SmoothSymbol<T> sy;
  for (int a = 0; a < 3; ++a) {
    sy.dk[a] = (T)((2.0 * M_PI) / ((double)p.nf[a] * p.h[a]));
    sy.n[a] = (T)p.desc.axis_n[a];
    sy.m[a] = (T)p.desc.axis_m[a];
  }
  const double* n = p.desc.axis_n;
  const double* m = p.desc.axis_m;
  sy.nm = (T)((n[0] * m[0] + n[1] * m[1]) + n[2] * m[2]);
  sy.inv_k02 = (T)(1.0 / (p.desc.split_k0 * p.desc.split_k0));
  sy.scale = (T)(1.0 / ((double)p.nf[0] * (double)p.nf[1] * (double)p.nf[2]));
  DDI_TRY((dispatch_policy<T, -1>(p.nf[0], PadX<T>{g, rho}, twiddles(p, p.nf[0]), s)));
  p.mark("smooth_pad_fft_x", s);
  DDI_TRY((dispatch_policy<T, -1>(p.nf[1], BlockY<T, true>{g}, twiddles(p, p.nf[1]), s)));
  p.mark("smooth_fft_y_fwd", s);
  DDI_TRY((dispatch_policy<T, -1>(p.nf[2], SmoothZ<T>{g, sy}, twiddles(p, p.nf[2]), s)));
  p.mark("smooth_fft_z_symbol", s);
  DDI_TRY((dispatch_policy<T, +1>(p.nf[2], AllZ<T, false>{g}, twiddles(p, p.nf[2]), s)));
  p.mark("smooth_fft_z_inv", s);
  DDI_TRY((dispatch_policy<T, +1>(p.nf[1], BlockY<T, false>{g}, twiddles(p, p.nf[1]), s)));
  p.mark("smooth_fft_y_inv", s);
  DDI_TRY((dispatch_policy<T, +1>(p.nf[0], CropX<T, false>{g, phi}, twiddles(p, p.nf[0]), s)));
  p.mark("smooth_fft_x_inv_crop", s);
  return DDI_OK;
}

template int nufft_forward_fft<float>(Plan&, const float*, cudaStream_t);
template int nufft_forward_fft<double>(Plan&, const double*, cudaStream_t);
template int nufft_inverse_fft<float>(Plan&, float*, cudaStream_t, bool);
template int nufft_inverse_fft<double>(Plan&, double*, cudaStream_t, bool);
template int split_smooth_part<float>(Plan&, const float*, float*, cudaStream_t);
template int split_smooth_part<double>(Plan&, const double*, double*, cudaStream_t);

}  // namespace ddi

// Fine-grid FFTs of the NUFFT with the zero padding and the cropping built in.
//
// The type-2 input occupies the n^d centred positions j' mod nf (j' = -n/2..n/2-1) of the
// 2n-oversampled grid and the type-1 output is read back at the same positions, so:
//   forward  x: only the n^(d-1) rows through the padded block exist; their input is
//               rho / psihat read straight from rho (pad and deconvolution fused);
//            y: only the planes z in the block; elements outside the block read as zero;
//            z: every column; elements outside the block read as zero.
//   inverse  z: every column; only the z in the block are stored;
//            y: only the planes z in the block; only the y in the block are stored;
//            x: only the rows in the block; the x in the block are stored as
//               Re(u) / psihat into phi (crop, deconvolution and real part fused).
// The NUFFT passes run once per evaluation and use the twiddles' FP32 heads only (the
// path's error budget is 1e-6); the GPE's repeated transforms use heads and tails.
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
  const T* dcx;
  const T* dcy;
  const T* dcz;
  C* fine;
  __device__ long long fidx(int lz, int ly, int lx) const {
    return ((long long)lz * ay.nf + ly) * ax.nf + lx;
  }
};

// forward x with the pad: lines = grid rows (jy, jz)
template <typename T>
struct RowRef {
  long long grid;  // offset of the row in rho / phi
  long long fine;  // offset of the row in the fine grid
  T dy, dz;        // deconvolution factors of the row
};

template <typename T>
struct PadX {
  using C = cx_t<T>;
  using Ref = RowRef<T>;
  static constexpr bool kPreciseTwiddles = false;
  Geo<T> g;
  const T* rho;
  __host__ __device__ long long nlines() const { return (long long)g.ay.n * g.az.n; }
  __device__ bool contig() const { return true; }
  __device__ Ref ref(long long L) const {
    const int jy = (int)(L % g.ay.n), jz = (int)(L / g.ay.n);
    return Ref{L * g.ax.n, g.fidx(g.az.fine_of(jz), g.ay.fine_of(jy), 0), g.dcy[jy], g.dcz[jz]};
  }
  __device__ C load(const Ref& r, int i) const {
    if (!g.ax.in_block(i)) return cmk<C>((T)0, (T)0);
    const int jx = g.ax.grid_of(i);
    return cmk<C>(__ldg(rho + r.grid + jx) * (g.dcx[jx] * r.dy * r.dz), (T)0);
  }
  __device__ void store(const Ref& r, int i, C v) const { g.fine[r.fine + i] = v; }
};

// y lines of the planes z in the block: forward (pruned input) or inverse (pruned output)
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
    if (FWD && !g.ay.in_block(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + r + (long long)i * g.ax.nf);
  }
  __device__ void store(Ref r, int i, C v) const {
    if (!FWD && !g.ay.in_block(i)) return;
    g.fine[r + (long long)i * g.ax.nf] = v;
  }
};

// z columns: forward (pruned input) or inverse (pruned output)
template <typename T, bool FWD>
struct AllZ {
  using C = cx_t<T>;
  static constexpr bool kPreciseTwiddles = false;
  using Ref = long long;  // the column's (y, x) offset
  Geo<T> g;
  __host__ __device__ long long nlines() const { return (long long)g.ax.nf * g.ay.nf; }
  __device__ bool contig() const { return false; }
  __device__ Ref ref(long long L) const { return L; }
  __device__ C load(Ref r, int i) const {
    if (FWD && !g.az.in_block(i)) return cmk<C>((T)0, (T)0);
    return __ldg(g.fine + (long long)i * g.ay.nf * g.ax.nf + r);
  }
  __device__ void store(Ref r, int i, C v) const {
    if (!FWD && !g.az.in_block(i)) return;
    g.fine[(long long)i * g.ay.nf * g.ax.nf + r] = v;
  }
};

// inverse x with crop, deconvolution and real part: lines = grid rows (jy, jz)
template <typename T>
struct CropX {
  using C = cx_t<T>;
  using Ref = RowRef<T>;
  static constexpr bool kPreciseTwiddles = false;
  Geo<T> g;
  T* phi;
  __host__ __device__ long long nlines() const { return (long long)g.ay.n * g.az.n; }
  __device__ bool contig() const { return true; }
  __device__ Ref ref(long long L) const {
    const int jy = (int)(L % g.ay.n), jz = (int)(L / g.ay.n);
    return Ref{L * g.ax.n, g.fidx(g.az.fine_of(jz), g.ay.fine_of(jy), 0), g.dcy[jy], g.dcz[jz]};
  }
  __device__ C load(const Ref& r, int i) const { return __ldg(g.fine + r.fine + i); }
  __device__ void store(const Ref& r, int i, C v) const {
    if (!g.ax.in_block(i)) return;
    const int jx = g.ax.grid_of(i);
    phi[r.grid + jx] = v.x * (g.dcx[jx] * r.dy * r.dz);
  }
};

template <typename T>
Geo<T> geo_of(Plan& p) {
  Geo<T> g;
  g.ax = Axis{p.n[0], p.nf[0]};
  g.ay = Axis{p.n[1], p.nf[1]};
  g.az = Axis{p.n[2], p.nf[2]};
  const T* dc = static_cast<const T*>(p.d_deconv);
  g.dcx = dc;
  g.dcy = dc + p.n[0];
  g.dcz = dc + p.n[0] + p.n[1];
  g.fine = static_cast<cx_t<T>*>(p.d_fine);
  return g;
}

}  // namespace

template <typename T>
int nufft_forward_fft(Plan& p, const T* rho, cudaStream_t s) {
  const Geo<T> g = geo_of<T>(p);
  DDI_TRY((dispatch_policy<T, -1>(p.nf[0], PadX<T>{g, rho}, twiddles(p, p.nf[0]), s)));
  p.mark("pad_fft_x", s);
  DDI_TRY((dispatch_policy<T, -1>(p.nf[1], BlockY<T, true>{g}, twiddles(p, p.nf[1]), s)));
  p.mark("fft_y_fwd", s);
  if (p.dim == 3) {
    DDI_TRY((dispatch_policy<T, -1>(p.nf[2], AllZ<T, true>{g}, twiddles(p, p.nf[2]), s)));
    p.mark("fft_z_fwd", s);
  }
  return DDI_OK;
}

template <typename T>
int nufft_inverse_fft(Plan& p, T* phi, cudaStream_t s) {
  const Geo<T> g = geo_of<T>(p);
  if (p.dim == 3) {
    DDI_TRY((dispatch_policy<T, +1>(p.nf[2], AllZ<T, false>{g}, twiddles(p, p.nf[2]), s)));
    p.mark("fft_z_inv", s);
  }
  DDI_TRY((dispatch_policy<T, +1>(p.nf[1], BlockY<T, false>{g}, twiddles(p, p.nf[1]), s)));
  p.mark("fft_y_inv", s);
  DDI_TRY((dispatch_policy<T, +1>(p.nf[0], CropX<T>{g, phi}, twiddles(p, p.nf[0]), s)));
  p.mark("fft_x_inv_crop", s);
  return DDI_OK;
}

template int nufft_forward_fft<float>(Plan&, const float*, cudaStream_t);
template int nufft_forward_fft<double>(Plan&, const double*, cudaStream_t);
template int nufft_inverse_fft<float>(Plan&, float*, cudaStream_t);
template int nufft_inverse_fft<double>(Plan&, double*, cudaStream_t);

}  // namespace ddi

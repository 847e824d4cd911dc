// GPE layer on top of the DDI: time-splitting Fourier pseudospectral step (Sec. 4.1,
// Eq. tssp2, Case I), energies (Sec. 3.2), normalised gradient flow with backward
// Euler (Sec. 3.1, Eqs. gf-eq2..gffg33) and the adjoint of one TSFP step.
//
// Grids are the plan's n[0] x n[1] x n[2] periodic box; Fourier modes are
// mu_p = 2 pi p / len, p = -n/2..n/2-1 (stored in FFT order).  The FFTs of fft.cu are
// unnormalised, so every Fourier-space multiplier below carries the 1/N_tot factor.
// Reductions accumulate in FP64 per thread, per block (fixed order), then one block
// sums the block partials in a fixed order: results are deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace ddi {
namespace {

constexpr int kThreads = 256;
constexpr int kRedMax = 8;  // sums per reduction

struct G3 {
  int n[3];
  double len[3];
  double ks[3];  // 2 pi / len: mode p has wavenumber p ks
};

G3 g3_of(const Plan& p) {
  G3 g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = p.n[d];
    g.len[d] = p.desc.len[d] > 0 ? p.desc.len[d] : 1.0;
    g.ks[d] = 2.0 * M_PI / g.len[d];
  }
  return g;
}

__device__ __forceinline__ double mode_mu(int l, int n, double ks) {
  const int pp = l < n / 2 ? l : l - n;
  return (double)pp * ks;
}

// grids hold < 2^31 points (at most 512^3 in 3D), so 32-bit index arithmetic suffices
__device__ __forceinline__ void idx3(long long idx, const G3& g, int& x, int& y, int& z) {
  const unsigned i = (unsigned)idx, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
  const unsigned r = i / n0;
  x = (int)(i - r * n0);
  z = (int)(r / n1);
  y = (int)(r - (unsigned)z * n1);
}

// e^{ia} - 1 = (-2 sin^2(a/2), sin a), accurate also when a is small.  A phase factor is
// applied as v + v (e^{ia} - 1): in FP32 a rounded e^{ia} near 1 cannot have |e| = 1 (the
// grid below 1 is 6e-8 apart), and a fixed |e| != 1 per mode or grid point would change
// the mass by the same amount every step; applied this way only the unbiased rounding
// of the result remains.
template <typename T>
__device__ __forceinline__ cx_t<T> expm1_i(T a) {
  T s, c;
  if constexpr (sizeof(T) == 4) {
    sincosf(0.5f * a, &s, &c);
  } else {
    sincos(0.5 * a, &s, &c);
  }
  return cmk<cx_t<T>>((T)-2 * s * s, (T)2 * s * c);
}

// per-axis factors e^{i f mu_d^2} - 1 (FP64 built, rounded once) for separable kinetic phases
template <typename T>
__global__ void k_phase_tables(cx_t<T>* tab, G3 g, double f) {
  const int total = g.n[0] + g.n[1] + g.n[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int d = 0, l = i;
    while (l >= g.n[d]) {
      l -= g.n[d];
      ++d;
    }
    const double mu = g.n[d] == 1 ? 0.0 : mode_mu(l, g.n[d], g.ks[d]);
    double s, c;
    sincos(0.5 * f * mu * mu, &s, &c);
    tab[i] = cmk<cx_t<T>>((T)(-2.0 * s * s), (T)(2.0 * s * c));
  }
}

// v * k for a constant known in FP64: head + tail in FP32 (a rounded 1/N would scale the
// state by the same wrong factor every step)
template <typename T>
__device__ __forceinline__ T scale_const(T v, double k) {
  if constexpr (sizeof(T) == 4) {
    const float hi = (float)k;
    return fmaf(v, hi, v * (float)(k - (double)hi));
  } else {
    return v * (T)k;
  }
}

// psihat <- psihat * e^{i f |mu|^2} / N_tot using the per-axis tables of e - 1:
// (1+A)(1+B)(1+C) - 1 = P + C + C P with P = A + B + A B
template <typename T>
__global__ void k_kinetic(cx_t<T>* __restrict__ a, const cx_t<T>* __restrict__ tab, G3 g, double inv_n) {
  using C = cx_t<T>;
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  const C* tx = tab;
  const C* ty = tab + g.n[0];
  const C* tz = ty + g.n[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    idx3(i, g, x, y, z);
    const C A = tx[x], B = ty[y], Cz = tz[z];
    const C P = cadd(cadd(A, B), cmul(A, B));
    const C E = cadd(cadd(P, Cz), cmul(Cz, P));
    const C v = a[i];
    const C r = cadd(v, cmul(v, E));
    a[i] = cmk<C>(scale_const(r.x, inv_n), scale_const(r.y, inv_n));
  }
}

template <typename T>
__global__ void k_abs2(const cx_t<T>* __restrict__ psi, T* __restrict__ rho, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const cx_t<T> v = psi[i];
    rho[i] = v.x * v.x + v.y * v.y;
  }
}

// ---- general nonlinearity and damping (Sec. 5, Eqs. DipGPE1, tssp2, fun1, fun2) -----------
// On the nonlinear sub-step |psi|^2 = h(phi, tau) obeys dh/dtau = -2 f(h) h; the step is
// psi2 = psi1 exp(-i [dt V + H + lambda U_dip * g]) exp(-F) with, for phi = |psi1|^2,
// H = beta int_0^dt h^sigma, F = int_0^dt f(h), g = int_0^dt h, in closed form for
// f = 0 (Case I), f = delta (Case II), f = delta rho^q (Case III).
struct NonlinParams {
  double sigma, delta, q;
  int damping;          // 0, 1 (linear), 2 (power)
  double c2_h, c2_g;    // Case II: (1 - e^{-2 delta sigma dt}) / (2 delta sigma), (1 - e^{-2 delta dt}) / (2 delta)
};

template <typename T>
__device__ __forceinline__ T powt(T a, T b) {
  if constexpr (sizeof(T) == 4) return powf(a, b); else return pow(a, b);
}
template <typename T>
__device__ __forceinline__ T log1pt(T a) {
  if constexpr (sizeof(T) == 4) return log1pf(a); else return log1p(a);
}
template <typename T>
__device__ __forceinline__ T expm1t(T a) {
  if constexpr (sizeof(T) == 4) return expm1f(a); else return expm1(a);
}

// g(phi) = int_0^dt h(phi, tau) d tau, the density whose DDI is G / lambda
template <typename T>
__global__ void k_step_density(const cx_t<T>* __restrict__ psi, T* __restrict__ gout, NonlinParams nl, T dt,
                               long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const cx_t<T> v = psi[i];
    const T phi = v.x * v.x + v.y * v.y;
    T g;
    if (nl.damping == 0) {
      g = dt * phi;
    } else if (nl.damping == 1) {
      g = (T)nl.c2_g * phi;
    } else {
      const T q = (T)nl.q, delta = (T)nl.delta;
      const T L = log1pt((T)2 * q * delta * dt * powt(phi, q));
      if (nl.q == 1.0) {
        g = L / ((T)2 * delta);
      } else {
        g = phi > (T)0 ? expm1t(((T)1 - (T)1 / q) * L) / ((T)2 * delta * (q - (T)1) * powt(phi, q - (T)1)) : (T)0;
      }
    }
    gout[i] = g;
  }
}

// psi <- psi exp(-i [dt V + H(phi) + lambda Phi_g]) exp(-F(phi)), phi = |psi|^2
template <typename T>
__global__ void k_nonlinear_general(cx_t<T>* __restrict__ psi, const T* __restrict__ V, const T* __restrict__ phig,
                                    T beta, T lam, T dt, NonlinParams nl, long long total) {
  using C = cx_t<T>;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const C v = psi[i];
    const T phi = v.x * v.x + v.y * v.y;
    const T sig = (T)nl.sigma;
    const T ps = nl.sigma == 1.0 ? phi : powt(phi, sig);
    T H, F;
    if (nl.damping == 0) {
      H = beta * ps * dt;
      F = (T)0;
    } else if (nl.damping == 1) {
      H = beta * ps * (T)nl.c2_h;
      F = (T)nl.delta * dt;
    } else {
      const T q = (T)nl.q, delta = (T)nl.delta;
      const T L = log1pt((T)2 * q * delta * dt * powt(phi, q));
      F = L / ((T)2 * q);
      if (nl.sigma == nl.q) {
        H = beta * L / ((T)2 * q * delta);
      } else {
        H = phi > (T)0 ? beta * powt(phi, sig - q) / ((T)2 * delta * (q - sig)) * expm1t(((T)1 - sig / q) * L) : (T)0;
      }
    }
    const T th = dt * V[i] + H + lam * phig[i];
    const C r = cadd(v, cmul(v, expm1_i(-th)));
    const T amp = nl.damping == 0 ? (T)1 : (sizeof(T) == 4 ? (T)expf((float)-F) : (T)exp((double)-F));
    psi[i] = cmk<C>(r.x * amp, r.y * amp);
  }
}

// psi <- psi exp(-i dt (V + beta rho + lambda Phi)), rho = |psi|^2 (Case I of Eq. tssp2)
template <typename T>
__global__ void k_nonlinear(cx_t<T>* __restrict__ psi, const T* __restrict__ V, const T* __restrict__ rho,
                            const T* __restrict__ phi, T beta, T lam, T dt, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const T th = V[i] + beta * rho[i] + lam * phi[i];
    const cx_t<T> v = psi[i];
    psi[i] = cadd(v, cmul(v, expm1_i(-dt * th)));
  }
}

// ---- FP64 reductions ------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* out) {
  __shared__ double sh[kRedMax][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += sh[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
}

template <int K>
__device__ __forceinline__ void block_max(double (&v)[K], double* out) {
  __shared__ double sh[kRedMax][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = -INFINITY;
    for (int w = 0; w < kThreads / 32; ++w) s = fmax(s, sh[threadIdx.x][w]);
    out[threadIdx.x] = s;
  }
}

// sums over the grid: mass, V|psi|^2, |psi|^4, Phi|psi|^2 (Phi may be null)
template <typename T>
__global__ void k_red_energy(const cx_t<T>* __restrict__ psi, const T* __restrict__ V,
                             const T* __restrict__ phi, long long total, double* part) {
  double v[4] = {0, 0, 0, 0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const cx_t<T> a = psi[i];
    const double r = (double)a.x * a.x + (double)a.y * a.y;
    v[0] += r;
    v[1] += (double)V[i] * r;
    v[2] += r * r;
    if (phi) v[3] += (double)phi[i] * r;
  }
  block_sum<4>(v, part + (size_t)blockIdx.x * kRedMax);
}

// sum |mu|^2 |psihat|^2
template <typename T>
__global__ void k_red_kinetic(const cx_t<T>* __restrict__ a, G3 g, double* part) {
  double v[1] = {0};
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    idx3(i, g, x, y, z);
    double m2 = 0.0;
    if (g.n[0] > 1) { const double m = mode_mu(x, g.n[0], g.ks[0]); m2 += m * m; }
    if (g.n[1] > 1) { const double m = mode_mu(y, g.n[1], g.ks[1]); m2 += m * m; }
    if (g.n[2] > 1) { const double m = mode_mu(z, g.n[2], g.ks[2]); m2 += m * m; }
    const cx_t<T> c = a[i];
    v[0] += m2 * ((double)c.x * c.x + (double)c.y * c.y);
  }
  block_sum<1>(v, part + (size_t)blockIdx.x * kRedMax);
}

// max and -min of W = V + beta |psi|^2 + lambda Phi, and a NaN/Inf flag
template <typename T>
__global__ void k_red_wrange(const T* __restrict__ V, const T* __restrict__ rho, const T* __restrict__ phi,
                             double beta, double lam, long long total, double* part) {
  double v[3] = {-INFINITY, -INFINITY, 0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double w = (double)V[i] + beta * (double)rho[i] + (phi ? lam * (double)phi[i] : 0.0);
    if (!isfinite(w)) v[2] = 1.0;
    v[0] = fmax(v[0], w);
    v[1] = fmax(v[1], -w);
  }
  block_max<3>(v, part + (size_t)blockIdx.x * kRedMax);
}

// max |a - b| and max |a|
template <typename T>
__global__ void k_red_maxdiff(const cx_t<T>* __restrict__ a, const cx_t<T>* __restrict__ b, long long total,
                              double* part) {
  // maxima of |a - b|^2 and |a|^2 in the working precision (the caller takes the roots);
  // a non-finite difference counts as infinite
  T m[2] = {(T)0, (T)0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const cx_t<T> x = a[i], y = b[i];
    const T dr = x.x - y.x, di = x.y - y.y;
    const T d2 = dr * dr + di * di;
    m[0] = isfinite(d2) ? (d2 > m[0] ? d2 : m[0]) : (T)INFINITY;
    const T a2 = x.x * x.x + x.y * x.y;
    m[1] = a2 > m[1] ? a2 : m[1];
  }
  double v[2] = {(double)m[0], (double)m[1]};
  block_max<2>(v, part + (size_t)blockIdx.x * kRedMax);
}

__global__ void __launch_bounds__(256) k_red_final(const double* part, int blocks, int k, int is_max, double* out) {
  // 256 threads: thread t folds partials t, t + 256, ... in index order, then a fixed
  // shared-memory tree combines the threads (deterministic)
  __shared__ double sh[kRedMax][256];
  const int t = threadIdx.x;
  for (int q = 0; q < k; ++q) {
    double s = is_max ? -INFINITY : 0.0;
    for (int b = t; b < blocks; b += 256) {
      const double x = part[(size_t)b * kRedMax + q];
      s = is_max ? fmax(s, x) : s + x;
    }
    sh[q][t] = s;
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w)
      for (int q = 0; q < k; ++q) sh[q][t] = is_max ? fmax(sh[q][t], sh[q][t + w]) : sh[q][t] + sh[q][t + w];
    __syncthreads();
  }
  if (t < k) out[t] = sh[t][0];
}

// GF: rhs = phi/dt + (alpha - W) cur, W = V + beta rho + lambda Phi
template <typename T>
__global__ void k_gf_rhs(const cx_t<T>* __restrict__ phi, const cx_t<T>* __restrict__ cur,
                         const T* __restrict__ V, const T* __restrict__ rho, const T* __restrict__ dip,
                         cx_t<T>* __restrict__ out, T beta, T lam, T alpha, T inv_dt, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const T w = V[i] + beta * rho[i] + (dip ? lam * dip[i] : (T)0);
    const T f = alpha - w;
    const cx_t<T> a = phi[i], c = cur[i];
    out[i] = cmk<cx_t<T>>(a.x * inv_dt + f * c.x, a.y * inv_dt + f * c.y);
  }
}

// GF: divide by (1/dt + alpha + |mu|^2/2) and by N_tot
template <typename T>
__global__ void k_gf_solve(cx_t<T>* __restrict__ a, G3 g, double inv_dt_alpha, double inv_n) {
  // in the working precision: the fixed point's own tolerance is the plan's (1e-7 in FP32)
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  const T ks[3] = {(T)g.ks[0], (T)g.ks[1], (T)g.ks[2]};
  const T c0 = (T)inv_dt_alpha, sc = (T)inv_n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int q[3];
    idx3(i, g, q[0], q[1], q[2]);
    T m2 = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int pp = q[d] < g.n[d] / 2 ? q[d] : q[d] - g.n[d];
      const T m = (T)pp * ks[d];
      m2 += g.n[d] > 1 ? m * m : (T)0;
    }
    const T f = sc / (c0 + (T)0.5 * m2);
    a[i] = cscale(a[i], f);
  }
}

template <typename T>
__global__ void k_scale(cx_t<T>* __restrict__ a, T s, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    a[i] = cscale(a[i], s);
}

// adjoint, part A: given psi1, rho = |psi1|^2, Phi, g2 (in cot):
//   e = exp(-i dt theta); r = Re(conj(-i dt psi1 e) g2); grad += dv r;
//   cot <- conj(e) g2; rout <- r
template <typename T>
__global__ void k_adj_a(const cx_t<T>* __restrict__ psi1, const T* __restrict__ V, const T* rho,
                        const T* __restrict__ phi, cx_t<T>* __restrict__ cot, T* __restrict__ grad,
                        T* rout, T beta, T lam, T dt, T dv, long long total) {
  using C = cx_t<T>;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const T th = V[i] + beta * rho[i] + lam * phi[i];
    const C em1 = expm1_i(-dt * th);  // e - 1, applied as in k_nonlinear
    const C v = psi1[i];
    const C psi2 = cadd(v, cmul(v, em1));
    // -i dt psi2 = dt (psi2.y, -psi2.x); Re(conj(u) g) = u.x g.x + u.y g.y
    const C g2 = cot[i];
    const T r = dt * (psi2.y * g2.x - psi2.x * g2.y);
    grad[i] += dv * r;
    rout[i] = r;
    cot[i] = cadd(g2, cmul(cconj(em1), g2));
  }
}

// adjoint, part B: cot += 2 psi1 (beta r + lambda Phi_r)
template <typename T>
__global__ void k_adj_b(const cx_t<T>* __restrict__ psi1, const T* __restrict__ r, const T* __restrict__ phir,
                        cx_t<T>* __restrict__ cot, T beta, T lam, long long total) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const T sfield = (T)2 * (beta * r[i] + (phir ? lam * phir[i] : (T)0));
    const cx_t<T> a = psi1[i], c = cot[i];
    cot[i] = cmk<cx_t<T>>(c.x + sfield * a.x, c.y + sfield * a.y);
  }
}

unsigned blocks_for(long long total) {
  long long b = (total + kThreads - 1) / kThreads;
  if (b > 152LL * 16) b = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

// ---- host helpers ------------------------------------------------------------------------------
// The observable of the trap-gradient problem, J = h^d sum_j x_j^2 |psi_j|^2 with x the
// coordinate along the grid's last axis (z in 3D, y in 2D), and its cotangent for the real
// pairing Re h^d sum conj(a) b: dJ/dpsi = 2 x^2 psi (written to cot when it is not null).
template <typename T>
__global__ void k_observable(const cx_t<T>* __restrict__ psi, cx_t<T>* __restrict__ cot, G3 g, int last, double lo,
                             double h, double* part) {
  double v[1] = {0.0};
  const long long total = (long long)g.n[0] * g.n[1] * g.n[2];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    idx3(i, g, x, y, z);
    const int j = last == 2 ? z : (last == 1 ? y : x);
    const double c = lo + (double)j * h;
    const cx_t<T> a = psi[i];
    v[0] += c * c * ((double)a.x * a.x + (double)a.y * a.y);
    if (cot) cot[i] = cmk<cx_t<T>>((T)(2.0 * c * c) * a.x, (T)(2.0 * c * c) * a.y);
  }
  block_sum<1>(v, part + (size_t)blockIdx.x * kRedMax);
}

template <typename T>
struct Gpe {
  using C = cx_t<T>;
  Plan& p;
  cudaStream_t s;
  long long N;
  G3 g;

  Gpe(Plan& pl, cudaStream_t st) : p(pl), s(st), N(pl.grid_points()), g(g3_of(pl)) {}

  int fft(C* a, int dir) { return fft_3d<T>(p, a, p.n[0], p.n[1], p.n[2], dir, s); }

  // a <- F^{-1} e^{i f |mu|^2} F a
  int kinetic(C* a, double f) {
    DDI_TRY(fft(a, -1));
    C* tab = static_cast<C*>(p.d_kin);
    k_phase_tables<T><<<4, kThreads, 0, s>>>(tab, g, f);
    DDI_LAUNCH_CHECK();
    k_kinetic<T><<<blocks_for(N), kThreads, 0, s>>>(a, tab, g, 1.0 / (double)N);
    DDI_LAUNCH_CHECK();
    return fft(a, +1);
  }

  int abs2(const C* a, T* out) {
    k_abs2<T><<<blocks_for(N), kThreads, 0, s>>>(a, out, N);
    DDI_LAUNCH_CHECK();
    return DDI_OK;
  }

  int reduce(int k, int is_max, double* host_out) {
    k_red_final<<<1, 256, 0, s>>>(p.d_red, p.red_blocks, k, is_max, p.d_red + (size_t)p.red_blocks * kRedMax);
    DDI_LAUNCH_CHECK();
    DDI_CUDA(cudaMemcpyAsync(p.h_red, p.d_red + (size_t)p.red_blocks * kRedMax, sizeof(double) * k,
                             cudaMemcpyDeviceToHost, s));
    DDI_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < k; ++i) host_out[i] = p.h_red[i];
    return DDI_OK;
  }

  int energy(const C* psi, const T* V, double beta, double lam, gpe_stats* out) {
    // Phi of |psi|^2 (skipped when lambda = 0)
    DDI_TRY(abs2(psi, static_cast<T*>(p.d_rho)));
    const T* phi = nullptr;
    if (lam != 0.0) {
      DDI_TRY(run_ddi<T>(p, static_cast<const T*>(p.d_rho), static_cast<T*>(p.d_phi), s));
      phi = static_cast<const T*>(p.d_phi);
    }
    k_red_energy<T><<<p.red_blocks, kThreads, 0, s>>>(psi, V, phi, N, p.d_red);
    DDI_LAUNCH_CHECK();
    double sums[4];
    DDI_TRY(reduce(4, 0, sums));
    C* w = static_cast<C*>(p.d_work2);
    DDI_CUDA(cudaMemcpyAsync(w, psi, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
    DDI_TRY(fft(w, -1));
    k_red_kinetic<T><<<p.red_blocks, kThreads, 0, s>>>(w, g, p.d_red);
    DDI_LAUNCH_CHECK();
    double kin;
    DDI_TRY(reduce(1, 0, &kin));
    const double dv = p.dv;
    out->mass = dv * sums[0];
    out->Ekin = 0.5 * dv / (double)N * kin;
    out->Epot = dv * sums[1];
    out->Eint = 0.5 * beta * dv * sums[2];
    out->Edip = lam != 0.0 ? 0.5 * lam * dv * sums[3] : 0.0;
    out->E = out->Ekin + out->Epot + out->Eint + out->Edip;
    out->mu = out->E + out->Eint + out->Edip;
    out->virial = 2 * out->Ekin - 2 * out->Epot + 3 * out->Eint + 3 * out->Edip;
    if (!std::isfinite(out->E)) {
      set_error("energy is not finite");
      return DDI_ERR_NONFINITE;
    }
    return DDI_OK;
  }

  int normalise(C* a, double* mass_out) {
    k_red_energy<T><<<p.red_blocks, kThreads, 0, s>>>(a, static_cast<const T*>(p.d_rho), nullptr, N, p.d_red);
    DDI_LAUNCH_CHECK();
    double sums[4];
    DDI_TRY(reduce(1, 0, sums));
    const double m = p.dv * sums[0];
    if (!(m > 0.0) || !std::isfinite(m)) {
      set_error("state has zero or non-finite mass");
      return DDI_ERR_NONFINITE;
    }
    k_scale<T><<<blocks_for(N), kThreads, 0, s>>>(a, (T)(1.0 / std::sqrt(m)), N);
    DDI_LAUNCH_CHECK();
    if (mass_out) *mass_out = m;
    return DDI_OK;
  }

  int maxdiff(const C* a, const C* b, double* d, double* amax) {
    k_red_maxdiff<T><<<p.red_blocks, kThreads, 0, s>>>(a, b, N, p.d_red);
    DDI_LAUNCH_CHECK();
    double v[2];
    DDI_TRY(reduce(2, 1, v));  // maxima of the squares
    *d = std::sqrt(v[0]);
    if (amax) *amax = std::sqrt(v[1]);
    return DDI_OK;
  }

  int step(C* psi, const T* V, double beta, double lam, double dt, int nsteps) {
    T* rho = static_cast<T*>(p.d_rho);
    T* phi = static_cast<T*>(p.d_phi);
    // consecutive half kinetic steps merge into one full step between nonlinear steps
    DDI_TRY(kinetic(psi, -0.25 * dt));
    for (int k = 0; k < nsteps; ++k) {
      DDI_TRY(abs2(psi, rho));
      if (lam != 0.0) {
        DDI_TRY(run_ddi<T>(p, rho, phi, s));
      } else {
        DDI_CUDA(cudaMemsetAsync(phi, 0, sizeof(T) * N, s));
      }
      k_nonlinear<T><<<blocks_for(N), kThreads, 0, s>>>(psi, V, rho, phi, (T)beta, (T)lam, (T)dt, N);
      DDI_LAUNCH_CHECK();
      DDI_TRY(kinetic(psi, k + 1 < nsteps ? -0.5 * dt : -0.25 * dt));
    }
    return DDI_OK;
  }

  // Eq. tssp2 for Eq. DipGPE1 (general nonlinearity and damping, fixed axis)
  int step_general(C* psi, const T* V, double beta, double lam, const NonlinParams& nl, double dt, int nsteps) {
    T* g = static_cast<T*>(p.d_rho);
    T* phi = static_cast<T*>(p.d_phi);
    DDI_TRY(kinetic(psi, -0.25 * dt));
    for (int k = 0; k < nsteps; ++k) {
      k_step_density<T><<<blocks_for(N), kThreads, 0, s>>>(psi, g, nl, (T)dt, N);
      DDI_LAUNCH_CHECK();
      if (lam != 0.0) {
        DDI_TRY(run_ddi<T>(p, g, phi, s));
      } else {
        DDI_CUDA(cudaMemsetAsync(phi, 0, sizeof(T) * N, s));
      }
      k_nonlinear_general<T><<<blocks_for(N), kThreads, 0, s>>>(psi, V, phi, (T)beta, (T)lam, (T)dt, nl, N);
      DDI_LAUNCH_CHECK();
      DDI_TRY(kinetic(psi, k + 1 < nsteps ? -0.5 * dt : -0.25 * dt));
    }
    return DDI_OK;
  }

  // J of the state psi (FP64 reduction; synchronises) and, when cot is not null, its cotangent
  int observable(const C* psi, C* cot, double* J) {
    const int last = p.dim - 1;
    k_observable<T><<<p.red_blocks, kThreads, 0, s>>>(psi, cot, g, last, p.desc.lo[last], p.h[last], p.d_red);
    DDI_LAUNCH_CHECK();
    double sum = 0.0;
    DDI_TRY(reduce(1, 0, &sum));
    *J = p.dv * sum;
    if (!std::isfinite(*J)) {
      set_error("the observable is not finite");
      return DDI_ERR_NONFINITE;
    }
    return DDI_OK;
  }

  // states kept by trap_gradient: checkpoints every `every` steps, then one segment's step inputs
  static size_t trap_states(int nsteps, int every) { return (size_t)((nsteps + every - 1) / every) + (size_t)every; }

  // nsteps single Strang steps from psi0 into cur (cur != psi0), then J; the forward run alone
  int trap_forward(const C* psi0, C* cur, const T* V, double beta, double lam, double dt, int nsteps, double* J) {
    DDI_CUDA(cudaMemcpyAsync(cur, psi0, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < nsteps; ++k) DDI_TRY(step(cur, V, beta, lam, dt, 1));
    return observable(cur, nullptr, J);
  }

  // J after nsteps steps and dJ/dV by the hand-written adjoint of each step, with
  // checkpointed recomputation: the forward sweep keeps the state every `every` steps, the
  // backward sweep recomputes each segment's step inputs from its checkpoint and applies the
  // step adjoints in reverse.  work: trap_states(nsteps, every) + 2 states.
  int trap_gradient(const C* psi0, const T* V, double beta, double lam, double dt, int nsteps, int every, C* work,
                    double* J, T* grad) {
    const int ncp = (nsteps + every - 1) / every;
    C* ckpt = work;                               // [ncp]
    C* seg = work + (size_t)ncp * N;              // [every]: one segment's step inputs
    C* cur = seg + (size_t)every * N;             // the running state
    C* cot = cur + N;                             // the cotangent
    DDI_CUDA(cudaMemcpyAsync(cur, psi0, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < nsteps; ++k) {
      if (k % every == 0) DDI_CUDA(cudaMemcpyAsync(ckpt + (size_t)(k / every) * N, cur, sizeof(C) * N,
                                                   cudaMemcpyDeviceToDevice, s));
      DDI_TRY(step(cur, V, beta, lam, dt, 1));
    }
    DDI_TRY(observable(cur, cot, J));
    DDI_CUDA(cudaMemsetAsync(grad, 0, sizeof(T) * N, s));
    for (int c = ncp - 1; c >= 0; --c) {
      const int k0 = c * every, k1 = std::min(nsteps, k0 + every);
      DDI_CUDA(cudaMemcpyAsync(seg, ckpt + (size_t)c * N, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
      for (int k = k0 + 1; k < k1; ++k) {
        C* prev = seg + (size_t)(k - 1 - k0) * N;
        C* next = prev + N;
        DDI_CUDA(cudaMemcpyAsync(next, prev, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
        DDI_TRY(step(next, V, beta, lam, dt, 1));
      }
      for (int k = k1 - 1; k >= k0; --k) DDI_TRY(adjoint(seg + (size_t)(k - k0) * N, cot, grad, V, beta, lam, dt));
    }
    return DDI_OK;
  }

  int adjoint(const C* psi_in, C* cot, T* grad, const T* V, double beta, double lam, double dt) {
    C* psi1 = static_cast<C*>(p.d_psi1);
    T* rho = static_cast<T*>(p.d_rho);
    T* phi = static_cast<T*>(p.d_phi);
    DDI_CUDA(cudaMemcpyAsync(psi1, psi_in, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
    DDI_TRY(kinetic(psi1, -0.25 * dt));
    DDI_TRY(abs2(psi1, rho));
    if (lam != 0.0) {
      DDI_TRY(run_ddi<T>(p, rho, phi, s));
    } else {
      DDI_CUDA(cudaMemsetAsync(phi, 0, sizeof(T) * N, s));
    }
    DDI_TRY(kinetic(cot, +0.25 * dt));
    k_adj_a<T><<<blocks_for(N), kThreads, 0, s>>>(psi1, V, rho, phi, cot, grad, rho, (T)beta, (T)lam, (T)dt,
                                                  (T)p.dv, N);
    DDI_LAUNCH_CHECK();
    if (lam != 0.0) DDI_TRY(run_ddi<T>(p, rho, phi, s));
    k_adj_b<T><<<blocks_for(N), kThreads, 0, s>>>(psi1, rho, lam != 0.0 ? phi : nullptr, cot, (T)beta, (T)lam, N);
    DDI_LAUNCH_CHECK();
    return kinetic(cot, +0.25 * dt);
  }

  int ground_state(C* phi0, const T* V, double beta, double lam, double dt, double tol, int rule,
                   double inner_tol, int max_steps, int check_every, gpe_stats* out) {
    C* cur = static_cast<C*>(p.d_psi1);
    C* nxt = static_cast<C*>(p.d_work);
    C* prev = static_cast<C*>(p.d_work2);
    T* rho = static_cast<T*>(p.d_rho);
    T* dip = static_cast<T*>(p.d_phi);
    DDI_TRY(normalise(phi0, nullptr));
    gpe_stats st{};
    DDI_TRY(energy(phi0, V, beta, lam, &st));
    double e_prev = st.E;
    int inner_max_seen = 0;
    double change = INFINITY;
    if (check_every < 1) check_every = 1;
    for (int n = 1; n <= max_steps; ++n) {
      // W = V + beta |phi|^2 + lambda Phi(|phi|^2) and alpha = (max W + min W) / 2
      DDI_TRY(abs2(phi0, rho));
      if (lam != 0.0) DDI_TRY(run_ddi<T>(p, rho, dip, s));
      k_red_wrange<T><<<p.red_blocks, kThreads, 0, s>>>(V, rho, lam != 0.0 ? dip : nullptr, beta, lam, N, p.d_red);
      DDI_LAUNCH_CHECK();
      double wr[3];
      DDI_TRY(reduce(3, 1, wr));
      if (wr[2] > 0.0) {
        set_error("non-finite effective potential at gradient-flow step %d", n);
        return DDI_ERR_NONFINITE;
      }
      const double alpha = 0.5 * (wr[0] - wr[1]);
      const double inv_dt_alpha = 1.0 / dt + alpha;
      DDI_CUDA(cudaMemcpyAsync(cur, phi0, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
      int it = 0;
      for (it = 1; it <= 200; ++it) {
        k_gf_rhs<T><<<blocks_for(N), kThreads, 0, s>>>(phi0, cur, V, rho, lam != 0.0 ? dip : nullptr, nxt, (T)beta,
                                                       (T)lam, (T)alpha, (T)(1.0 / dt), N);
        DDI_LAUNCH_CHECK();
        DDI_TRY(fft(nxt, -1));
        k_gf_solve<T><<<blocks_for(N), kThreads, 0, s>>>(nxt, g, inv_dt_alpha, 1.0 / (double)N);
        DDI_LAUNCH_CHECK();
        DDI_TRY(fft(nxt, +1));
        double d;
        DDI_TRY(maxdiff(nxt, cur, &d, nullptr));
        C* t = cur;
        cur = nxt;
        nxt = t;
        if (!std::isfinite(d)) {
          set_error("gradient-flow inner iteration diverged at step %d", n);
          return DDI_ERR_NONFINITE;
        }
        if (d <= inner_tol) break;
      }
      if (it > 200) it = 200;
      inner_max_seen = it > inner_max_seen ? it : inner_max_seen;
      DDI_TRY(normalise(cur, nullptr));
      // cur is phi^{n+1}; keep phi^n in prev for the paper's rule
      DDI_CUDA(cudaMemcpyAsync(prev, phi0, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
      DDI_CUDA(cudaMemcpyAsync(phi0, cur, sizeof(C) * N, cudaMemcpyDeviceToDevice, s));
      if (n % check_every == 0 || n == max_steps) {
        bool done;
        if (rule == GPE_STOP_PAPER) {
          double d;
          DDI_TRY(maxdiff(phi0, prev, &d, nullptr));
          change = d / dt;
          done = change <= tol;
        } else {
          DDI_TRY(energy(phi0, V, beta, lam, &st));
          change = std::fabs(st.E - e_prev);
          e_prev = st.E;
          done = change < tol;
        }
        if (done) {
          DDI_TRY(energy(phi0, V, beta, lam, &st));
          st.steps = n;
          st.inner_max = inner_max_seen;
          st.last_change = change;
          *out = st;
          return DDI_OK;
        }
      }
    }
    DDI_TRY(energy(phi0, V, beta, lam, &st));
    st.steps = max_steps;
    st.inner_max = inner_max_seen;
    st.last_change = change;
    *out = st;
    set_error("gradient flow did not reach tol %.3g in %d steps (last change %.3g)", tol, max_steps, change);
    return DDI_ERR_NOCONV;
  }
};

int check_gpe(ddi_plan plan, const void* a, const void* b) {
  if (!plan || !a || !b) {
    set_error("plan and array pointers must not be NULL");
    return DDI_ERR_ARG;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->p.device) {
    set_error("the current device is not the plan's device");
    return DDI_ERR_ARG;
  }
  return DDI_OK;
}

bool finite_params(std::initializer_list<double> v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

}  // namespace
}  // namespace ddi

using ddi::Gpe;

extern "C" {

int gpe_step(ddi_plan plan, void* psi, const void* V, double beta, double lambda, double dt, int nsteps,
             void* stream) {
  return ddi::guarded("gpe_step", [&]() -> int {
    DDI_TRY(ddi::check_gpe(plan, psi, V));
    if (nsteps < 0 || !ddi::finite_params({beta, lambda, dt})) {
      ddi::set_error("nsteps must be >= 0 and beta, lambda, dt finite");
      return DDI_ERR_ARG;
    }
    if (nsteps == 0) return DDI_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->p.prec == DDI_FP64) {
      Gpe<double> g(plan->p, s);
      return g.step(static_cast<double2*>(psi), static_cast<const double*>(V), beta, lambda, dt, nsteps);
    }
    Gpe<float> g(plan->p, s);
    return g.step(static_cast<float2*>(psi), static_cast<const float*>(V), beta, lambda, dt, nsteps);
  });
}

int gpe_step_ex(ddi_plan plan, void* psi, const void* V, double beta, double lambda, const gpe_nonlinearity* nl,
                double dt, int nsteps, void* stream) {
  return ddi::guarded("gpe_step_ex", [&]() -> int {
    DDI_TRY(ddi::check_gpe(plan, psi, V));
    if (!nl || nsteps < 0 || !ddi::finite_params({beta, lambda, dt, nl->sigma, nl->delta, nl->q}) ||
        !(nl->sigma > 0.0) || nl->damping < GPE_DAMP_NONE || nl->damping > GPE_DAMP_POWER ||
        (nl->damping != GPE_DAMP_NONE && !(nl->delta > 0.0)) || (nl->damping == GPE_DAMP_POWER && !(nl->q > 0.0))) {
      ddi::set_error("gpe_step_ex: nl must not be NULL, nsteps >= 0, parameters finite, sigma > 0, damping one of "
                     "GPE_DAMP_*, delta > 0 when damped, q > 0 for GPE_DAMP_POWER");
      return DDI_ERR_ARG;
    }
    if (nsteps == 0) return DDI_OK;
    ddi::NonlinParams np{nl->sigma, nl->delta, nl->q, nl->damping, 0.0, 0.0};
    if (nl->damping == GPE_DAMP_LINEAR) {
      np.c2_h = -std::expm1(-2.0 * nl->delta * nl->sigma * dt) / (2.0 * nl->delta * nl->sigma);
      np.c2_g = -std::expm1(-2.0 * nl->delta * dt) / (2.0 * nl->delta);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->p.prec == DDI_FP64) {
      Gpe<double> g(plan->p, s);
      return g.step_general(static_cast<double2*>(psi), static_cast<const double*>(V), beta, lambda, np, dt, nsteps);
    }
    Gpe<float> g(plan->p, s);
    return g.step_general(static_cast<float2*>(psi), static_cast<const float*>(V), beta, lambda, np, dt, nsteps);
  });
}

int gpe_energy(ddi_plan plan, const void* psi, const void* V, double beta, double lambda, gpe_stats* out,
               void* stream) {
  return ddi::guarded("gpe_energy", [&]() -> int {
    DDI_TRY(ddi::check_gpe(plan, psi, V));
    if (!out || !ddi::finite_params({beta, lambda})) {
      ddi::set_error("out must not be NULL and beta, lambda finite");
      return DDI_ERR_ARG;
    }
    memset(out, 0, sizeof *out);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->p.prec == DDI_FP64) {
      Gpe<double> g(plan->p, s);
      return g.energy(static_cast<const double2*>(psi), static_cast<const double*>(V), beta, lambda, out);
    }
    Gpe<float> g(plan->p, s);
    return g.energy(static_cast<const float2*>(psi), static_cast<const float*>(V), beta, lambda, out);
  });
}

int gpe_ground_state(ddi_plan plan, void* phi, const void* V, double beta, double lambda, double dt, double tol,
                     int rule, double inner_tol, int max_steps, int check_every, gpe_stats* out, void* stream) {
  return ddi::guarded("gpe_ground_state", [&]() -> int {
    DDI_TRY(ddi::check_gpe(plan, phi, V));
    if (!out || !(dt > 0.0) || !(tol > 0.0) || !(inner_tol > 0.0) || max_steps < 1 ||
        (rule != GPE_STOP_ENERGY && rule != GPE_STOP_PAPER) || !ddi::finite_params({beta, lambda, dt, tol})) {
      ddi::set_error("invalid gradient-flow arguments (dt, tol, inner_tol > 0; max_steps >= 1; rule 0/1)");
      return DDI_ERR_ARG;
    }
    memset(out, 0, sizeof *out);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->p.prec == DDI_FP64) {
      Gpe<double> g(plan->p, s);
      return g.ground_state(static_cast<double2*>(phi), static_cast<const double*>(V), beta, lambda, dt, tol, rule,
                            inner_tol, max_steps, check_every, out);
    }
    Gpe<float> g(plan->p, s);
    return g.ground_state(static_cast<float2*>(phi), static_cast<const float*>(V), beta, lambda, dt, tol, rule,
                          inner_tol, max_steps, check_every, out);
  });
}

int gpe_step_adjoint(ddi_plan plan, const void* psi_in, void* cot, void* grad_V, const void* V, double beta,
                     double lambda, double dt, void* stream) {
  return ddi::guarded("gpe_step_adjoint", [&]() -> int {
    DDI_TRY(ddi::check_gpe(plan, psi_in, cot));
    DDI_TRY(ddi::check_gpe(plan, grad_V, V));
    if (!ddi::finite_params({beta, lambda, dt})) {
      ddi::set_error("beta, lambda, dt must be finite");
      return DDI_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->p.prec == DDI_FP64) {
      Gpe<double> g(plan->p, s);
      return g.adjoint(static_cast<const double2*>(psi_in), static_cast<double2*>(cot), static_cast<double*>(grad_V),
                       static_cast<const double*>(V), beta, lambda, dt);
    }
    Gpe<float> g(plan->p, s);
    return g.adjoint(static_cast<const float2*>(psi_in), static_cast<float2*>(cot), static_cast<float*>(grad_V),
                     static_cast<const float*>(V), beta, lambda, dt);
  });
}

int gpe_trap_observable(ddi_plan plan, const void* psi0, const void* V, double beta, double lambda, double dt,
                        int nsteps, void* psi_T, double* J, void* stream) {
  return ddi::guarded("gpe_trap_observable", [&]() -> int {
    DDI_TRY(ddi::check_gpe(plan, psi0, V));
    DDI_TRY(ddi::check_gpe(plan, psi_T, V));
    if (!J || nsteps < 0 || psi_T == psi0 || !ddi::finite_params({beta, lambda, dt})) {
      ddi::set_error("gpe_trap_observable: J must not be NULL, psi_T must differ from psi0, nsteps >= 0, "
                     "beta, lambda, dt finite");
      return DDI_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->p.prec == DDI_FP64) {
      Gpe<double> g(plan->p, s);
      return g.trap_forward(static_cast<const double2*>(psi0), static_cast<double2*>(psi_T),
                            static_cast<const double*>(V), beta, lambda, dt, nsteps, J);
    }
    Gpe<float> g(plan->p, s);
    return g.trap_forward(static_cast<const float2*>(psi0), static_cast<float2*>(psi_T), static_cast<const float*>(V),
                          beta, lambda, dt, nsteps, J);
  });
}

int gpe_trap_gradient_workspace(ddi_plan plan, int nsteps, int checkpoint, size_t* bytes) {
  return ddi::guarded("gpe_trap_gradient_workspace", [&]() -> int {
    if (!plan || !bytes || nsteps < 1 || checkpoint < 1) {
      ddi::set_error("gpe_trap_gradient_workspace: plan and bytes must not be NULL, nsteps and checkpoint >= 1");
      return DDI_ERR_ARG;
    }
    const size_t states = Gpe<double>::trap_states(nsteps, checkpoint) + 2;
    *bytes = states * (size_t)plan->p.grid_points() * plan->p.cx_size();
    return DDI_OK;
  });
}

int gpe_trap_gradient(ddi_plan plan, const void* psi0, const void* V, double beta, double lambda, double dt,
                      int nsteps, int checkpoint, void* work, size_t work_bytes, double* J, void* grad_V,
                      void* stream) {
  return ddi::guarded("gpe_trap_gradient", [&]() -> int {
    DDI_TRY(ddi::check_gpe(plan, psi0, V));
    DDI_TRY(ddi::check_gpe(plan, work, grad_V));
    size_t need = 0;
    if (!J || nsteps < 1 || checkpoint < 1 || !ddi::finite_params({beta, lambda, dt})) {
      ddi::set_error("gpe_trap_gradient: J must not be NULL, nsteps and checkpoint >= 1, beta, lambda, dt finite");
      return DDI_ERR_ARG;
    }
    DDI_TRY(gpe_trap_gradient_workspace(plan, nsteps, checkpoint, &need));
    if (work_bytes < need) {
      ddi::set_error("gpe_trap_gradient: workspace of %zu bytes, %zu needed", work_bytes, need);
      return DDI_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->p.prec == DDI_FP64) {
      Gpe<double> g(plan->p, s);
      return g.trap_gradient(static_cast<const double2*>(psi0), static_cast<const double*>(V), beta, lambda, dt,
                             nsteps, checkpoint, static_cast<double2*>(work), J, static_cast<double*>(grad_V));
    }
    Gpe<float> g(plan->p, s);
    return g.trap_gradient(static_cast<const float2*>(psi0), static_cast<const float*>(V), beta, lambda, dt, nsteps,
                           checkpoint, static_cast<float2*>(work), J, static_cast<float*>(grad_V));
  });
}

}  // extern "C"

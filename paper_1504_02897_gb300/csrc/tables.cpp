// Quadrature tables of Sec. 2.1 (Eq. DDI-Trun1), built on the host in FP64.
//
// Every expression is written in a fixed evaluation order using +, -, *, / and sqrt
// after the libm cos/sin calls (and exp, for the window of split plans), and this file is
// compiled with -ffp-contract=off, so the tables are reproducible bit for bit by any
// implementation of the same rule on the same libm.
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace ddi {

namespace {
const double kTwoPi = 2.0 * M_PI;

// grid sizes the FFTs support: 2^a or 3 * 2^a (a >= 2)
bool valid_n(int v) {
  if (v < 8 || (v % 4) != 0) return false;
  int odd = v / (v & (-v));
  return odd == 1 || odd == 3;
}

void legendre(int n, double z, double* p_out, double* dp_out) {
  double p0 = 1.0, p1 = z;
  for (int k = 1; k < n; ++k) {
    double p2 = ((double)(2 * k + 1) * z * p1 - (double)k * p0) / (double)(k + 1);
    p0 = p1;
    p1 = p2;
  }
  *p_out = p1;
  *dp_out = ((double)n * (z * p1 - p0)) / (z * z - 1.0);
}
}  // namespace

void gauss_legendre(int n, double* x, double* w) {
  // Newton on the Legendre recurrence from cos(pi (i + 3/4) / (n + 1/2)), stopped when
  // the update is exactly zero or after 100 updates; weight 2 / ((1 - x^2) P_n'(x)^2).
  const int half = (n + 1) / 2;
  for (int i = 0; i < half; ++i) {
    double z;
    if (n % 2 == 1 && i == half - 1) {
      z = 0.0;  // the middle root of an odd rule is exactly zero
    } else {
      z = std::cos((M_PI * ((double)i + 0.75)) / ((double)n + 0.5));
      int iters = 0;
      for (;;) {
        double p, dp;
        legendre(n, z, &p, &dp);
        double dz = p / dp;
        z = z - dz;
        ++iters;
        if (dz == 0.0 || iters >= 100) break;
      }
    }
    double p, dp;
    legendre(n, z, &p, &dp);
    double wt = 2.0 / (((1.0 - z * z) * dp) * dp);
    x[n - 1 - i] = z;
    x[i] = -z;
    w[n - 1 - i] = wt;
    w[i] = wt;
  }
}

int normalise_desc(const ddi_plan_desc* in, ddi_plan_desc* out, std::string* err) {
  char buf[256];
  if (!in) {
    *err = "descriptor is NULL";
    return DDI_ERR_ARG;
  }
  *out = *in;
  ddi_plan_desc& d = *out;
  if (d.dim != 2 && d.dim != 3) {
    *err = "dim must be 2 or 3";
    return DDI_ERR_ARG;
  }
  if (d.dim == 2) d.n[2] = 1;
  const int nmax_axis = d.dim == 3 ? 512 : 1024;
  for (int a = 0; a < d.dim; ++a) {
    if (!valid_n(d.n[a]) || d.n[a] > nmax_axis) {
      snprintf(buf, sizeof buf, "n[%d] = %d: grid sizes must be 2^a or 3 * 2^a in [8, %d]", a, d.n[a],
               nmax_axis);
      *err = buf;
      return DDI_ERR_ARG;
    }
    if (!(d.len[a] > 0.0) || !std::isfinite(d.len[a]) || !std::isfinite(d.lo[a])) {
      snprintf(buf, sizeof buf, "len[%d] must be finite and > 0, lo finite", a);
      *err = buf;
      return DDI_ERR_ARG;
    }
  }
  auto norm3 = [](const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); };
  double nn = norm3(d.axis_n);
  if (!(std::fabs(nn - 1.0) <= 1e-9)) {
    snprintf(buf, sizeof buf, "axis_n must be a unit vector (|n| = %.17g)", nn);
    *err = buf;
    return DDI_ERR_ARG;
  }
  if (d.axis_m[0] == 0.0 && d.axis_m[1] == 0.0 && d.axis_m[2] == 0.0) {
    for (int a = 0; a < 3; ++a) d.axis_m[a] = d.axis_n[a];
  }
  double mm = norm3(d.axis_m);
  if (!(std::fabs(mm - 1.0) <= 1e-9)) {
    snprintf(buf, sizeof buf, "axis_m must be a unit vector (|m| = %.17g)", mm);
    *err = buf;
    return DDI_ERR_ARG;
  }
  int nmax = 0;
  for (int a = 0; a < d.dim; ++a) nmax = d.n[a] > nmax ? d.n[a] : nmax;
  if (!std::isfinite(d.split_k0)) {
    *err = "split_k0 must be finite";
    return DDI_ERR_ARG;
  }
  if (d.split_k0 != 0.0) {
    // the split algorithm of Sec. 2.1 (Eq. 3.9): window width, ball radius and ball rule
    if (d.dim != 3) {
      *err = "the split algorithm (split_k0 != 0) is built for 3D plans";
      return DDI_ERR_ARG;
    }
    if (d.split_k0 < 0.0) {
      const double lmin = std::min(std::min(d.len[0], d.len[1]), d.len[2]);
      d.split_k0 = 9.6 / lmin;
    }
    if (d.kmax == 0.0) d.kmax = 6.0 * d.split_k0;
    const double diag = std::sqrt((d.len[0] * d.len[0] + d.len[1] * d.len[1]) + d.len[2] * d.len[2]);
    const double K = d.kmax * diag;
    auto size_for = [](double v, int least) {
      const double c = std::ceil(std::min(v, 1e6) / 8.0) * 8.0;
      return c < (double)least ? least : (int)c;
    };
    if (d.nr == 0) d.nr = size_for(0.48 * K, 16);
    if (d.ntheta == 0) d.ntheta = size_for(0.32 * K, 8);
    if (d.nphi == 0) d.nphi = size_for(0.64 * K, 16);
  }
  if (d.spread != DDI_SPREAD_AUTO && d.spread != DDI_SPREAD_TILES && d.spread != DDI_SPREAD_COLUMNS) {
    *err = "spread must be DDI_SPREAD_AUTO, DDI_SPREAD_TILES or DDI_SPREAD_COLUMNS";
    return DDI_ERR_ARG;
  }
  if (d.compensated != 0 && d.compensated != 1) {
    *err = "compensated must be 0 or 1";
    return DDI_ERR_ARG;
  }
  if (d.check_finite != 0 && d.check_finite != 1) {
    *err = "check_finite must be 0 or 1";
    return DDI_ERR_ARG;
  }
  if (d.split_full_passes != 0 && d.split_full_passes != 1) {
    *err = "split_full_passes must be 0 or 1";
    return DDI_ERR_ARG;
  }
  if (d.ellipsoid != 0 && d.ellipsoid != 1) {
    *err = "ellipsoid must be 0 or 1";
    return DDI_ERR_ARG;
  }
  if (d.ellipsoid && d.split_k0 != 0.0) {
    *err = "the ellipsoidal rule is not combined with the split algorithm";
    return DDI_ERR_ARG;
  }
  if (d.ellipsoid) {
    // the symbol at the direction of k turns over an angular band ~ min e / max e wide
    double hlo = 1e300, hhi = 0.0;
    for (int a = 0; a < d.dim; ++a) {
      const double h = d.len[a] / (double)d.n[a];
      hlo = h < hlo ? h : hlo;
      hhi = h > hhi ? h : hhi;
    }
    const double ratio = hhi / hlo;
    const double big = 1e6;
    if (d.dim == 3 && d.ntheta == 0) d.ntheta = (int)std::ceil(std::min(0.5 * nmax * ratio, big));
    if (d.dim == 2 && d.nphi == 0) d.nphi = 2 * (int)std::ceil(std::min(nmax * ratio, big));
  }
  if (d.dim == 3) {
    if (d.nr == 0) d.nr = nmax;
    if (d.ntheta == 0) d.ntheta = nmax / 2;
    if (d.nphi == 0) d.nphi = nmax;
  } else {
    if (d.nr == 0) d.nr = 2 * nmax;
    d.ntheta = 1;
    if (d.nphi == 0) d.nphi = 2 * nmax;
  }
  if (d.nr < 1 || d.nr > 8192 || d.ntheta < 1 || d.ntheta > 8192 || d.nphi < 2 || d.nphi > 16384 ||
      (d.nphi % 2) != 0) {
    *err = "quadrature sizes out of range (nr, ntheta in [1, 8192], nphi even in [2, 16384])";
    return DDI_ERR_ARG;
  }
  double hmin = 1e300;
  for (int a = 0; a < d.dim; ++a) {
    double h = d.len[a] / (double)d.n[a];
    hmin = h < hmin ? h : hmin;
  }
  if (d.kmax == 0.0) d.kmax = M_PI / hmin;
  if (!(d.kmax > 0.0) || !std::isfinite(d.kmax) || d.kmax > M_PI / hmin * (1.0 + 1e-12)) {
    *err = d.split_k0 != 0.0
               ? "kmax (default 6 split_k0) must be in (0, pi / min h]: refine the grid or give a smaller "
                 "split_k0 or kmax"
               : "kmax must be in (0, pi / min h]: the nodes must stay inside the fine grid's band";
    return DDI_ERR_ARG;
  }
  if (d.precision != DDI_FP64 && d.precision != DDI_FP32) {
    *err = "precision must be DDI_FP64 or DDI_FP32";
    return DDI_ERR_ARG;
  }
  if (d.nufft_tol == 0.0) d.nufft_tol = d.precision == DDI_FP64 ? 1e-13 : 1e-6;
  if (!(d.nufft_tol > 0.0) || d.nufft_tol >= 1e-2) {
    *err = "nufft_tol must be in (0, 1e-2)";
    return DDI_ERR_ARG;
  }
  int64_t M = (int64_t)d.nr * d.ntheta * d.nphi;
  if (M > (int64_t)1 << 30) {
    *err = "too many quadrature nodes (> 2^30)";
    return DDI_ERR_ARG;
  }
  return DDI_OK;
}

double symbol_divisor(int dim) { return dim == 3 ? (kTwoPi * kTwoPi) * kTwoPi : kTwoPi * kTwoPi; }

void build_quadrature(const ddi_plan_desc& d, QuadTables* t, bool keep_dirs) {
  t->dim = d.dim;
  for (int a = 0; a < 3; ++a) {
    t->n[a] = d.n[a];
    t->h[a] = d.len[a] / (double)d.n[a];
  }
  t->nr = d.nr;
  t->ntheta = d.ntheta;
  t->nphi = d.nphi;
  t->R = d.kmax;
  std::vector<double> xr(d.nr), wr0(d.nr);
  gauss_legendre(d.nr, xr.data(), wr0.data());
  const double half_R = 0.5 * t->R;
  std::vector<double> r(d.nr), wr(d.nr);
  for (int i = 0; i < d.nr; ++i) {
    r[i] = half_R * (1.0 + xr[i]);
    wr[i] = half_R * wr0[i];
  }
  const int half = d.nphi / 2;
  std::vector<double> c(d.nphi), s(d.nphi);
  for (int m = 0; m < half; ++m) {
    double ang = (kTwoPi * (double)m) / (double)d.nphi;
    c[m] = std::cos(ang);
    s[m] = std::sin(ang);
  }
  for (int m = 0; m < half; ++m) {
    c[half + m] = -c[m];
    s[half + m] = -s[m];
  }
  const double wphi = kTwoPi / (double)d.nphi;
  const double n0 = d.axis_n[0], n1 = d.axis_n[1], n2 = d.axis_n[2];
  const double m0 = d.axis_m[0], m1 = d.axis_m[1], m2 = d.axis_m[2];
  if (d.dim == 3) {
    std::vector<double> u(d.ntheta), wu(d.ntheta), st(d.ntheta);
    gauss_legendre(d.ntheta, u.data(), wu.data());
    for (int j = 0; j < d.ntheta; ++j) st[j] = std::sqrt((1.0 - u[j]) * (1.0 + u[j]));
    const double nm = (n0 * m0 + n1 * m1) + n2 * m2;
    const double tp3 = (kTwoPi * kTwoPi) * kTwoPi;
    // split plans (Eq. 3.9): every weight carries the window q(k) = exp(-|k|^2 / k0^2)
    const bool window = d.split_k0 > 0.0;
    const double k02 = d.split_k0 * d.split_k0;
    // ellipsoidal rule: nodes e * (r khat), Jacobian e_x e_y e_z, symbol at g / |g|, g = e * khat
    const bool ell = d.ellipsoid != 0;
    double e[3] = {1.0, 1.0, 1.0};
    if (ell) {
      double hmin = t->h[0];
      for (int a = 1; a < 3; ++a) hmin = t->h[a] < hmin ? t->h[a] : hmin;
      for (int a = 0; a < 3; ++a) e[a] = hmin / t->h[a];
    }
    const double J = (e[0] * e[1]) * e[2];
    t->M = (int64_t)d.nr * d.ntheta * d.nphi;
    t->k.resize(3 * t->M);
    t->W.resize(t->M);
    if (keep_dirs) t->dirw.resize(4 * t->M);
    int64_t q = 0;
    for (int i = 0; i < d.nr; ++i) {
      for (int j = 0; j < d.ntheta; ++j) {
        const double rst = r[i] * st[j];
        double wgt = ((wr[i] * wu[j]) * wphi) * (r[i] * r[i]);
        if (ell) wgt = wgt * J;
        for (int m = 0; m < d.nphi; ++m, ++q) {
          double hx, hy, hz;
          if (!ell) {
            t->k[3 * q + 0] = rst * c[m];
            t->k[3 * q + 1] = rst * s[m];
            t->k[3 * q + 2] = r[i] * u[j];
            hx = st[j] * c[m];
            hy = st[j] * s[m];
            hz = u[j];
          } else {
            t->k[3 * q + 0] = (rst * c[m]) * e[0];
            t->k[3 * q + 1] = (rst * s[m]) * e[1];
            t->k[3 * q + 2] = (r[i] * u[j]) * e[2];
            const double gx = (st[j] * c[m]) * e[0], gy = (st[j] * s[m]) * e[1], gz = u[j] * e[2];
            const double gn = std::sqrt((gx * gx + gy * gy) + gz * gz);
            hx = gx / gn;
            hy = gy / gn;
            hz = gz / gn;
          }
          const double nk = (n0 * hx + n1 * hy) + n2 * hz;
          const double mk = (m0 * hx + m1 * hy) + m2 * hz;
          const double sym = 3.0 * (nk * mk) - nm;
          double wq = wgt;
          if (window) {
            const double kx = t->k[3 * q + 0], ky = t->k[3 * q + 1], kz = t->k[3 * q + 2];
            wq = wgt * std::exp(-(((kx * kx + ky * ky) + kz * kz) / k02));
          }
          t->W[q] = (wq * sym) / tp3;
          if (keep_dirs) {
            double* o = &t->dirw[4 * q];
            o[0] = hx;
            o[1] = hy;
            o[2] = hz;
            o[3] = wq;
          }
        }
      }
    }
  } else {
    const double tp2 = kTwoPi * kTwoPi;
    t->M = (int64_t)d.nr * d.nphi;
    t->k.resize(2 * t->M);
    t->W.resize(t->M);
    if (keep_dirs) t->dirw.resize(4 * t->M);
    int64_t q = 0;
    // ellipsoidal rule: nodes e * (r khat), Jacobian e_x e_y, symbol factor |k| = r |g|,
    // symbol direction g / |g|, g = e * khat
    const bool ell = d.ellipsoid != 0;
    double e[2] = {1.0, 1.0};
    if (ell) {
      const double hmin = t->h[0] < t->h[1] ? t->h[0] : t->h[1];
      e[0] = hmin / t->h[0];
      e[1] = hmin / t->h[1];
    }
    const double J = e[0] * e[1];
    for (int i = 0; i < d.nr; ++i) {
      double wgt = (wr[i] * wphi) * (r[i] * r[i]);
      if (ell) wgt = wgt * J;
      for (int m = 0; m < d.nphi; ++m, ++q) {
        double hx = c[m], hy = s[m], wq = wgt;
        if (!ell) {
          t->k[2 * q + 0] = r[i] * c[m];
          t->k[2 * q + 1] = r[i] * s[m];
        } else {
          t->k[2 * q + 0] = (r[i] * c[m]) * e[0];
          t->k[2 * q + 1] = (r[i] * s[m]) * e[1];
          const double gx = c[m] * e[0], gy = s[m] * e[1];
          const double gn = std::sqrt(gx * gx + gy * gy);
          hx = gx / gn;
          hy = gy / gn;
          wq = wgt * gn;
        }
        const double nk = n0 * hx + n1 * hy;
        const double mk = m0 * hx + m1 * hy;
        const double sym = 1.5 * (nk * mk - n2 * m2);
        t->W[q] = (wq * sym) / tp2;
        if (keep_dirs) {
          double* o = &t->dirw[4 * q];
          o[0] = hx;
          o[1] = hy;
          o[2] = 0.0;
          o[3] = wq;
        }
      }
    }
  }
}

int kernel_width(const ddi_plan_desc& d) {
  // Exponential-of-semicircle kernel with 2x oversampling: the error falls roughly
  // as 10^{-(w - 1)} per NUFFT; two NUFFTs and the fine-grid FFTs consume some of the
  // budget, so one extra cell of width is kept.  Widths outside this set are not built.
  const double tol = d.nufft_tol;
  if (d.precision == DDI_FP32) return tol < 1e-5 ? 8 : 6;
  if (tol < 1e-13) return 16;
  if (tol < 1e-11) return 14;
  if (tol < 1e-9) return 12;
  return 10;
}

double kernel_beta(int width) { return 2.30 * (double)width; }

void split_band(const ddi_plan_desc& d, int width, int band[2]) {
  band[0] = band[1] = 0;
  if (!(d.split_k0 > 0.0) || d.split_full_passes || d.dim != 3) return;
  for (int a = 0; a < 2; ++a) {
    const double h = d.len[a] / (double)d.n[a];
    const int nf = 2 * d.n[a];
    const int b = (int)std::floor(d.kmax * h * (double)nf / kTwoPi + 0.5 * (double)width) + 2;
    band[a] = 2 * b + 1 < nf ? b : 0;
  }
  if (band[0] == 0 || band[1] == 0) band[0] = band[1] = 0;
}

int64_t fine_start(double k, double h, int nf, int width) {
  const double scale = (h * (double)nf) / kTwoPi;
  return (int64_t)std::ceil(k * scale - 0.5 * (double)width);
}

double es_kernel_hat(double xi, int width, double beta) {
  // (w/2) int_{-1}^{1} exp(beta (sqrt(1 - z^2) - 1)) cos(xi w z / 2) dz by 200-point
  // Gauss-Legendre; the integrand's endpoint behaviour is damped by exp(-beta).
  static thread_local std::vector<double> gx, gw;
  if (gx.empty()) {
    gx.resize(200);
    gw.resize(200);
    gauss_legendre(200, gx.data(), gw.data());
  }
  const double hw = 0.5 * (double)width;
  double acc = 0.0;
  for (int i = 0; i < 200; ++i) {
    const double z = gx[i];
    const double val = std::exp(beta * (std::sqrt((1.0 - z) * (1.0 + z)) - 1.0));
    acc += gw[i] * val * std::cos(xi * hw * z);
  }
  return hw * acc;
}

}  // namespace ddi

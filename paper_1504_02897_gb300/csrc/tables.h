// Host-side quadrature and NUFFT tables (FP64).  Built by tables.cpp, which is
// compiled by the host compiler with -ffp-contract=off so that every table is the
// exact result of the fixed evaluation order documented there.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ddi.h"

namespace ddi {

struct QuadTables {
  int dim = 3;
  int n[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  int nr = 0, ntheta = 1, nphi = 0;
  double R = 0.0;
  int64_t M = 0;
  std::vector<double> k;  // [M][dim]
  std::vector<double> W;  // [M]
  // [M][4], filled on request: what W is built from besides the axes, so that the
  // weights can be rebuilt for other axes (3D: unit direction hx, hy, hz and the weight
  // without the symbol; 2D: cos, sin, 0 and that weight)
  std::vector<double> dirw;
};

// Validates the descriptor and fills defaults; returns DDI_OK or DDI_ERR_ARG with *err set.
int normalise_desc(const ddi_plan_desc* in, ddi_plan_desc* out, std::string* err);

// Gauss-Legendre nodes (ascending) and weights on [-1, 1].
void gauss_legendre(int n, double* x, double* w);

// Quadrature nodes and DDI weights of Sec. 2.1 (Eq. DDI-Trun1) for a normalised descriptor.
void build_quadrature(const ddi_plan_desc& d, QuadTables* t, bool keep_dirs = false);
// (2 pi)^d, the divisor of W in build_quadrature, computed as it is there
double symbol_divisor(int dim);

// Fine-grid oversampling and kernel width for a normalised descriptor.
int kernel_width(const ddi_plan_desc& d);
double kernel_beta(int width);

// Split plans: half-widths (x, y) of the band of fine-grid lines around k = 0 that holds
// every tap of the ball's nodes, |l| <= kmax h nf / (2 pi) + w/2, plus two cells; 0 where the
// band would cover the axis, and both 0 when the plan does not split or asks for full passes.
void split_band(const ddi_plan_desc& d, int width, int band[2]);

// First fine-grid tap ceil(k * (h nf / 2pi) - w/2) along one axis.
int64_t fine_start(double k, double h, int nf, int width);

// Fourier transform of the exponential-of-semicircle kernel (fine-cell units),
// psihat(xi) = int_{-w/2}^{w/2} exp(beta (sqrt(1 - (2x/w)^2) - 1)) cos(xi x) dx.
double es_kernel_hat(double xi, int width, double beta);

}  // namespace ddi

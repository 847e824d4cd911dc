"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only (grids, densities, initial states, trap
perturbation directions); it contains none of the DDI/GPE arithmetic and is the one
module that both the CUDA-path tests and the CPU oracle tests draw inputs from.
Arrays are numpy, C-ordered [z][y][x] (3D) or [y][x] (2D).

Recipes (the paper uses analytic Gaussians and GPE states, no dataset):
* anisotropic_gaussian_density: rho = |psi|^2, psi = exp(-(x^2+y^2)/2 - z^2/(2*1.5^2))
  on [-L, L)^3, normalised to discrete mass h^3 sum rho = 1.
* gaussian_mixture_density: 8 axis-aligned Gaussians, per component (draw order):
  centre U[-4,4]^3, widths U[0.5,2]^3, amplitude U[0.5,1.5]; discrete mass 1.
* batch_2d: per density (draw order) N from {128,256,512,1024}, half-width L in U[8,16],
  tilt alpha in U[0,90] degrees, then 4 Gaussians with centre U[-L/2,L/2]^2,
  widths U[0.5,2]^2, amplitude U[0.5,1.5]; discrete mass 1; axis n = (sin a, 0, cos a).
* gpe_initial: trap Gaussian exp(-(g_x x^2 + g_y y^2 + g_z z^2)/2) times
  (1 + eps * eta), eta a smooth periodic field from 8 Fourier modes |p_d| <= 3 with
  N(0,1) cosine/sine coefficients scaled to max |eta| = 1; discrete mass 1.
* trap_directions: white noise N(0,1) smoothed by a Gaussian of width 2h (periodic),
  scaled to max |d| = 1.
* collapse_schedule: the time-dependent trap switch, beta(t) and lambda(t) of the
  collapse-and-explosion example of Sec. 5 (Example dy_app_damp).
"""
import math

import numpy as np


def box(N, L, dim=3):
    n = (N,) * dim
    return n, (-float(L),) * dim, (2.0 * L,) * dim


def coords(n, lo, length):
    """Coordinate arrays on the grid, returned as (X, Y[, Z]) broadcast to [z][y][x]."""
    dim = len(n)
    axes = [lo[d] + np.arange(n[d]) * (length[d] / n[d]) for d in range(dim)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return list(reversed(mesh))


def _normalise(rho, n, length):
    dv = float(np.prod([length[d] / n[d] for d in range(len(n))]))
    return rho / (dv * float(np.sum(rho))), dv


def anisotropic_gaussian_density(N=24, L=6.0):
    n, lo, ln = box(N, L)
    X, Y, Z = coords(n, lo, ln)
    raw = np.exp(-(X ** 2 + Y ** 2) - Z ** 2 / 2.25)
    rho, dv = _normalise(raw, n, ln)
    s2 = np.array([0.5, 0.5, 1.125])
    amp = rho.flat[0] / raw.flat[0] if raw.flat[0] > 0 else 1.0 / (dv * float(np.sum(raw)))
    mass = amp * float(np.prod(np.sqrt(2 * math.pi * s2)))
    return {"n": n, "lo": lo, "len": ln, "rho": rho, "s2": s2, "mass": mass,
            "axis": (0.0, 0.0, 1.0)}


def gaussian_mixture_density(N=128, L=12.0, seed=0, ngauss=8, dim=3, centre=4.0):
    rng = np.random.default_rng(seed)
    n, lo, ln = box(N, L, dim)
    X = coords(n, lo, ln)
    rho = np.zeros(X[0].shape)
    comps = []
    for _ in range(ngauss):
        c = rng.uniform(-centre, centre, dim)
        w = rng.uniform(0.5, 2.0, dim)
        a = rng.uniform(0.5, 1.5)
        expo = sum((X[d] - c[d]) ** 2 / (2 * w[d] ** 2) for d in range(dim))
        rho += a * np.exp(-expo)
        comps.append((a, w ** 2, c))
    rho, dv = _normalise(rho, n, ln)
    scale = 1.0 / (dv * float(np.sum(sum(
        a * np.exp(-sum((X[d] - c[d]) ** 2 / (2 * s2[d]) for d in range(dim))) for a, s2, c in comps))))
    mix = [(a * scale * float(np.prod(np.sqrt(2 * math.pi * s2))), s2, c) for a, s2, c in comps]
    alpha = math.radians(30.0)
    return {"n": n, "lo": lo, "len": ln, "rho": rho, "components": mix,
            "axis": (math.sin(alpha), 0.0, math.cos(alpha))}


def batch_2d(count=96, seed=0, sizes=(128, 256, 512, 1024), ngauss=4):
    rng = np.random.default_rng(seed)
    items = []
    for _ in range(count):
        N = int(sizes[rng.integers(0, len(sizes))])
        L = float(rng.uniform(8.0, 16.0))
        alpha = float(rng.uniform(0.0, 90.0))
        n, lo, ln = box(N, L, 2)
        X, Y = coords(n, lo, ln)
        rho = np.zeros(X.shape)
        for _ in range(ngauss):
            c = rng.uniform(-L / 2, L / 2, 2)
            w = rng.uniform(0.5, 2.0, 2)
            a = rng.uniform(0.5, 1.5)
            rho += a * np.exp(-((X - c[0]) ** 2 / (2 * w[0] ** 2) + (Y - c[1]) ** 2 / (2 * w[1] ** 2)))
        rho, _ = _normalise(rho, n, ln)
        ar = math.radians(alpha)
        items.append({"n": n, "lo": lo, "len": ln, "rho": rho, "alpha_deg": alpha,
                      "axis": (math.sin(ar), 0.0, math.cos(ar))})
    return items


def harmonic_trap(n, lo, length, gammas):
    """V = (sum_d gamma_d^2 x_d^2) / 2 (Eq. Vpoten)."""
    X = coords(n, lo, length)
    return 0.5 * sum((g * g) * X[d] ** 2 for d, g in enumerate(gammas))


def gpe_initial(n, lo, length, gammas, eps=0.0, seed=0, nmodes=8, pmax=3):
    X = coords(n, lo, length)
    dim = len(n)
    psi = np.exp(-0.5 * sum(g * X[d] ** 2 for d, g in enumerate(gammas)))
    if eps:
        rng = np.random.default_rng(seed)
        eta = np.zeros(X[0].shape)
        for _ in range(nmodes):
            p = rng.integers(-pmax, pmax + 1, dim)
            a, b = rng.standard_normal(2)
            arg = sum(2 * math.pi * p[d] * (X[d] - lo[d]) / length[d] for d in range(dim))
            eta += a * np.cos(arg) + b * np.sin(arg)
        eta /= np.max(np.abs(eta))
        psi = psi * (1.0 + eps * eta)
    dv = float(np.prod([length[d] / n[d] for d in range(dim)]))
    psi = psi / math.sqrt(dv * float(np.sum(psi * psi)))
    return psi.astype(np.complex128)


def trap_directions(n, count=16, seed=0):
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    out = []
    shape = tuple(reversed(n))
    for _ in range(count):
        d = ndimage.gaussian_filter(rng.standard_normal(shape), sigma=2.0, mode="wrap")
        out.append(d / np.max(np.abs(d)))
    return out


COLLAPSE_GAMMAS = (1.65, 1.0, 1.325)   # trap frequencies of Example dy_app_damp
COLLAPSE_BETA0 = 761.102


def collapse_b(t):
    """b(t) of Example dy_app_damp (t in [0, 1.2]), continuous at t = 0.4."""
    if t <= 0.4:
        return (-125.0 * t - 25.0 * math.exp(-5.0 * t) + 215.0) / 133.0
    return (25.0 * (1.0 - math.exp(-2.0)) * math.exp(-6.25 * t + 2.5) + 140.0) / 133.0


def collapse_schedule(t, t_hold=0.2):
    """(trap on, beta, lambda) at time t for Example dy_app_damp: the trap
    (gamma_x, gamma_y, gamma_z) = (1.65, 1, 1.325) is on for t <= 4 + t_hold, lambda = 82.864
    for t <= 5.6 + t_hold, and beta = 761.102 (1 + 28 / (75 t - 280)) on [0, 3.2], 761.102 * 0.3
    on [3.2, 3.6], 761.102 (1 - 1 / b(t - 3.6)) on [3.6, 4.8] and 38.8066 on [4.8, 5.6 + t_hold],
    then 0.  Reading: the printed formula multiplies every branch by 761.102, but the last
    nonzero branch is the value the third branch reaches at t = 4.8 (761.102 (1 - 1/b(1.2)) =
    38.807), so 38.8066 is beta itself, not a factor."""
    trap = t <= 4.0 + t_hold
    lam = 82.864 if t <= 5.6 + t_hold else 0.0
    if t <= 3.2:
        beta = COLLAPSE_BETA0 * (1.0 + 28.0 / (75.0 * t - 280.0))
    elif t <= 3.6:
        beta = COLLAPSE_BETA0 * 0.3
    elif t <= 4.8:
        beta = COLLAPSE_BETA0 * (1.0 - 1.0 / collapse_b(t - 3.6))
    elif t <= 5.6 + t_hold:
        beta = 38.8066
    else:
        beta = 0.0
    return trap, beta, lam


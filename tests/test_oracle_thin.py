"""Pins of the oracle's ellipsoidal rule for heterogeneous boxes (the thin domains D_eps of
Sec. 2.1, Tables ani_2d and ani_3d_cs1): with equal mesh sizes it is the spherical rule; on
thin boxes it reaches the closed forms of the z- (3D) and y-localised (2D) Gaussians of
Eqs. Coulomb:3D:aniso:z / DDI:2D:aniso (the oracle's 1-D integral forms) to the accuracy the
paper prints, where the spherical ball of radius pi / min h does not resolve the integrand."""
import math

import numpy as np

from oracle import closed_forms as cf
from oracle import nudft
from oracle import quadrature as qd

N_2D = np.array([0, -0.896, 0.44404]) / np.linalg.norm([0, -0.896, 0.44404])   # Example 2d_exmp
M_2D = np.array([0, -0.52476, 0.85125]) / np.linalg.norm([0, -0.52476, 0.85125])


def _thin_box(dim, L, eps, hx):
    n = (int(round(2 * L / hx)),) * dim
    lo = (-L,) * (dim - 1) + (-eps * L,)
    ln = (2 * L,) * (dim - 1) + (2 * eps * L,)
    ax = [lo[d] + np.arange(n[d]) * (ln[d] / n[d]) for d in range(dim)]
    mesh = list(reversed(np.meshgrid(*reversed(ax), indexing="ij")))
    pts = np.stack([g.ravel() for g in mesh], axis=1)
    return n, lo, ln, pts, mesh[0].shape


def test_equal_mesh_sizes_give_the_spherical_rule():
    for dim, n, ln, ax, m in [(3, (24, 24, 24), (12, 12, 12), (0.6, 0, 0.8), None),
                              (3, (16, 32, 8), (4, 8, 2), (0, 0, 1), (0.6, 0.8, 0)),
                              (2, (32, 32), (8, 8), N_2D, M_2D)]:
        a = qd.plan_tables(dim, n, ln, ax, m, nr=16, ntheta=12, nphi=24)
        b = qd.plan_tables(dim, n, ln, ax, m, nr=16, ntheta=12, nphi=24, ellipsoid=True)
        assert np.array_equal(a["k"], b["k"])
        # the symbol is formed from the normalised direction (|g| = 1 up to rounding), so W
        # agrees to roundoff of the largest weight (W itself cancels to ~0 on some directions)
        assert np.max(np.abs(a["W"] - b["W"])) <= 2e-15 * np.max(np.abs(a["W"]))


def test_thin_3d_box_matches_closed_form():
    # rho = exp(-(x^2+y^2)/4 - z^2/(4 eps^2)) / (8 pi^1.5 eps) (Eq. Coulomb:3D:aniso:z), n = m = z,
    # D_eps = [-8,8]^2 x [-2,2] (eps = 1/4), h_x = 1/2, h_z = eps h_x.  Table ani_3d_cs1 prints
    # 2.307e-8 for L = 8, eps = 1/4 (h_x = 1/4): the error at L = 8 is the density's truncation
    # at the box (exp(-16) of its peak); the ellipsoidal rule reaches that level
    eps = 0.25
    n, lo, ln, pts, shape = _thin_box(3, 8.0, eps, 0.5)
    s2 = [2.0, 2.0, 2.0 * eps * eps]
    rho = cf.gaussian_density(pts, s2, [0, 0, 0], 1.0).reshape(shape)
    nax = np.array([0.0, 0.0, 1.0])
    t = qd.plan_tables(3, n, ln, nax, nr=96, ntheta=48, nphi=96, ellipsoid=True)
    got = nudft.ddi(rho, t, n, lo, ln).ravel()
    sel = np.random.default_rng(0).choice(pts.shape[0], 300, replace=False)
    ex = cf.phi3d_gauss_integral(pts[sel], s2, [0, 0, 0], nax, None, mass=1.0)
    assert np.max(np.abs(got[sel] - ex)) / np.max(np.abs(ex)) <= 1e-7


def test_thin_3d_box_localised_in_two_directions():
    # the second kind of Eq. Coulomb:3D:aniso:xy: rho = exp(-(x^2+y^2)/(4 eps^2) - z^2/4) /
    # (8 pi^1.5 eps^2) on [-2,2]^2 x [-8,8] (eps = 1/4), h_x = h_y = eps h_z, h_z = 1/2: the
    # oblate ellipsoid resolves it to the same truncation level
    eps, L = 0.25, 8.0
    n = (32, 32, 32)
    lo = (-eps * L, -eps * L, -L)
    ln = (2 * eps * L, 2 * eps * L, 2 * L)
    ax = [lo[d] + np.arange(n[d]) * (ln[d] / n[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    s2 = [2.0 * eps * eps, 2.0 * eps * eps, 2.0]
    rho = cf.gaussian_density(pts, s2, [0, 0, 0], 1.0).reshape(X.shape)
    nax = np.array([0.0, 0.0, 1.0])
    t = qd.plan_tables(3, n, ln, nax, nr=96, ntheta=48, nphi=96, ellipsoid=True)
    got = nudft.ddi(rho, t, n, lo, ln).ravel()
    sel = np.random.default_rng(0).choice(pts.shape[0], 300, replace=False)
    ex = cf.phi3d_gauss_integral(pts[sel], s2, [0, 0, 0], nax, None, mass=1.0)
    assert np.max(np.abs(got[sel] - ex)) / np.max(np.abs(ex)) <= 1e-7


def test_thin_2d_box_matches_closed_form_to_the_papers_accuracy():
    # rho = exp(-x^2/4 - y^2/(4 eps^2)) / (4 pi eps) (Eq. Coulomb:2D:aniso), axes of Example
    # 2d_exmp, D_eps = [-16,16] x [-4,4] (eps = 1/4), h_x = 1/4, h_y = eps h_x.  Table ani_2d
    # prints 5.119e-15 for L = 16, eps = 1/4 (h_x = 1/8); the rule (default sizes) is within it
    eps = 0.25
    n, lo, ln, pts, shape = _thin_box(2, 16.0, eps, 0.25)
    s2 = [2.0, 2.0 * eps * eps]
    rho = cf.gaussian_density(pts, s2, [0, 0], 1.0).reshape(shape)
    t = qd.plan_tables(2, n, ln, N_2D, M_2D, ellipsoid=True)
    assert t["sizes"] == (256, 1, 1024)
    got = nudft.ddi(rho, t, n, lo, ln).ravel()
    sel = np.random.default_rng(0).choice(pts.shape[0], 300, replace=False)
    ex = cf.phi2d_gauss_integral(pts[sel], s2, [0, 0], N_2D, M_2D, mass=1.0)
    assert np.max(np.abs(got[sel] - ex)) / np.max(np.abs(ex)) <= 5.119e-15


def test_spherical_ball_does_not_resolve_a_thin_box():
    # why the reading exists: the ball of radius pi / h_y puts too few radial nodes where the
    # density's transform lives (|k_x| of order 1) to resolve e^{ik.x} across the long axis
    eps = 0.25
    n, lo, ln, pts, shape = _thin_box(2, 8.0, eps, 0.25)
    s2 = [2.0, 2.0 * eps * eps]
    rho = cf.gaussian_density(pts, s2, [0, 0], 1.0).reshape(shape)
    sel = np.random.default_rng(0).choice(pts.shape[0], 200, replace=False)
    ex = cf.phi2d_gauss_integral(pts[sel], s2, [0, 0], N_2D, M_2D, mass=1.0)
    errs = []
    for ell in (False, True):
        t = qd.plan_tables(2, n, ln, N_2D, M_2D, nr=128, nphi=512, ellipsoid=ell)
        got = nudft.ddi(rho, t, n, lo, ln).ravel()
        errs.append(np.max(np.abs(got[sel] - ex)) / np.max(np.abs(ex)))
    assert errs[0] > 1.0 and errs[1] < 1e-6

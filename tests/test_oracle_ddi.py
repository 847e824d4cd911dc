"""Pins of the oracle DDI (the discrete quadrature sum of Sec. 2.1) against things other
than itself: brute force, exact identities of the sum, and the paper's closed forms."""
import json
import math
import os

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import nudft
from oracle import quadrature as qd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _grid3(N, L):
    n = (N, N, N)
    lo = (-L, -L, -L)
    ln = (2 * L, 2 * L, 2 * L)
    ax = nudft.grid_axes(n, lo, ln)
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return n, lo, ln, X, Y, Z


def _rand_rho(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.random(shape)


def test_blocked_equals_bruteforce_3d():
    n, lo, ln = (5, 4, 6), (-1.0, -2.0, -1.5), (2.0, 4.0, 3.0)
    t = qd.plan_tables(3, n, ln, (0.5, 0.0, math.sqrt(0.75)), nr=3, ntheta=3, nphi=4)
    rho = _rand_rho((6, 4, 5), 1)
    a = nudft.ddi(rho, t, n, lo, ln)
    b = nudft.ddi_bruteforce(rho, t, n, lo, ln)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def test_blocked_equals_bruteforce_2d():
    n, lo, ln = (6, 5), (-2.0, -1.0), (3.0, 2.5)
    t = qd.plan_tables(2, n, ln, (0.3, 0.4, math.sqrt(0.75)), nr=4, nphi=6)
    rho = _rand_rho((5, 6), 2)
    a = nudft.ddi(rho, t, n, lo, ln)
    b = nudft.ddi_bruteforce(rho, t, n, lo, ln)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def test_sampled_equals_full():
    n, lo, ln, X, Y, Z = _grid3(10, 3.0)
    t = qd.plan_tables(3, n, ln, (0, 0, 1))
    rho = _rand_rho(X.shape, 3)
    full = nudft.ddi(rho, t, n, lo, ln)
    idx = np.array([[0, 0, 0], [9, 9, 9], [3, 5, 7], [2, 8, 1]])
    part = nudft.ddi_at(rho, t, n, lo, ln, idx)
    ref = full[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert np.max(np.abs(part - ref)) <= 1e-13 * np.max(np.abs(full))


def test_trace_identity():
    # Phi_{n=x} + Phi_{n=y} + Phi_{n=z} = 0 for any rho: the symbols sum to 3|khat|^2 - 3 = 0.
    n, lo, ln, X, Y, Z = _grid3(12, 4.0)
    rho = _rand_rho(X.shape, 4)
    tot = 0.0
    ref = None
    for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        t = qd.plan_tables(3, n, ln, e)
        phi = nudft.ddi(rho, t, n, lo, ln)
        ref = phi if ref is None else ref
        tot = tot + phi
    assert np.max(np.abs(tot)) <= 1e-13 * np.max(np.abs(ref))


def test_linearity():
    n, lo, ln, X, Y, Z = _grid3(10, 4.0)
    t = qd.plan_tables(3, n, ln, (0.5, 0, math.sqrt(0.75)))
    a = _rand_rho(X.shape, 5)
    b = _rand_rho(X.shape, 6)
    pa = nudft.ddi(a, t, n, lo, ln)
    pb = nudft.ddi(b, t, n, lo, ln)
    pab = nudft.ddi(2.0 * a - 3.0 * b, t, n, lo, ln)
    assert np.max(np.abs(pab - (2 * pa - 3 * pb))) <= 1e-13 * np.max(np.abs(pab))


def test_reflection_symmetry_about_dipole_axis():
    # n = z: reflecting rho in x (x -> -x on the symmetric part of the grid) reflects Phi,
    # because the node set is closed under k_x -> -k_x with equal weights.
    N, L = 12, 4.0
    n, lo, ln, X, Y, Z = _grid3(N, L)
    rng = np.random.default_rng(7)
    base = rng.random((N, N, N))
    base[:, :, 0] = 0.0
    base[:, 0, :] = 0.0
    base[0, :, :] = 0.0
    flip = np.zeros_like(base)
    flip[:, :, 1:] = base[:, :, 1:][:, :, ::-1]
    rho = base + flip                               # even in x (index j <-> N - j)
    t = qd.plan_tables(3, n, ln, (0, 0, 1))
    phi = nudft.ddi(rho, t, n, lo, ln)
    ref = phi[:, :, 1:][:, :, ::-1]
    assert np.max(np.abs(phi[:, :, 1:] - ref)) <= 1e-13 * np.max(np.abs(phi))
    # tilted axis in the x-z plane: y -> -y stays a symmetry
    rho_y = base + np.concatenate([np.zeros((N, 1, N)), base[:, 1:, :][:, ::-1, :]], axis=1)
    t = qd.plan_tables(3, n, ln, (0.5, 0, math.sqrt(0.75)))
    phi = nudft.ddi(rho_y, t, n, lo, ln)
    assert np.max(np.abs(phi[:, 1:, :] - phi[:, 1:, :][:, ::-1, :])) <= 1e-13 * np.max(np.abs(phi))


def test_parseval_energy_identity():
    # h^3 sum_j rho_j Phi_j = sum_q W_q |rhohat_q|^2: type 1 is the adjoint of type 2.
    n, lo, ln, X, Y, Z = _grid3(10, 4.0)
    t = qd.plan_tables(3, n, ln, (0.5, 0, math.sqrt(0.75)))
    rho = _rand_rho(X.shape, 8)
    phi = nudft.ddi(rho, t, n, lo, ln)
    lhs = (8.0 / 10) ** 3 * float(np.sum(rho * phi))
    rh = nudft.type2(rho, t["k"], n, lo, ln)
    rhs = float(np.sum(t["W"] * np.abs(rh) ** 2))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_type2_of_gaussian_matches_fourier_transform():
    # rhohat_q of a well-resolved Gaussian equals its continuous Fourier transform
    # (f^(k) = int f e^{-i k.x} dx, Eq. DipKer convention) to spectral accuracy, on nodes
    # with |k| <= R/2 (closer to pi/h the trapezoid sum aliases, by design of the rule).
    n, lo, ln, X, Y, Z = _grid3(40, 10.0)
    s2 = np.array([1.0, 1.2, 1.5])
    rho = np.exp(-(X ** 2 / (2 * s2[0]) + Y ** 2 / (2 * s2[1]) + Z ** 2 / (2 * s2[2])))
    mass = float(np.prod(np.sqrt(2 * math.pi * s2)))
    t = qd.plan_tables(3, n, ln, (0, 0, 1), nr=6, ntheta=3, nphi=4)
    k = t["k"]
    sel = np.linalg.norm(k, axis=1) <= t["R"] / 2
    rh = nudft.type2(rho, k[sel], n, lo, ln)
    exact = mass * np.exp(-0.5 * np.sum(k[sel] * k[sel] * s2, axis=1))
    assert sel.sum() >= 12
    assert np.max(np.abs(rh - exact)) <= 1e-12 * mass


def _phi3_exact(X, Y, Z, sigma, n, m=None):
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    ex = cf.phi3d_erf(pts, sigma, n, m)
    r = np.linalg.norm(pts, axis=1)
    small = r < 0.1          # the Erf form cancels catastrophically near r = 0
    if small.any():
        ex[small] = cf.phi3d_gauss_integral(pts[small], [sigma ** 2 / 2] * 3, [0, 0, 0], n, m,
                                            mass=(math.pi * sigma ** 2) ** 1.5)
    return ex.reshape(X.shape)


def test_closed_forms_agree_3d():
    # The paper's Erf/Hessian closed form (Eqs. extDensGausDipolar, Hessian_Ex1) and the
    # 1-D integral derived from the symbol are independent formulas for the same Phi.
    rng = np.random.default_rng(0)
    x = rng.uniform(-4, 4, (30, 3))
    sig = 1.4
    tab = json.load(open(GOLDEN))["tab:diff:dip"]["setup"]
    n = np.array(tab["n"]); n /= np.linalg.norm(n)
    m = np.array(tab["m"]); m /= np.linalg.norm(m)
    for nn, mm in ((n, m), (np.array([0, 0, 1.0]), None)):
        a = cf.phi3d_erf(x, sig, nn, mm)
        b = cf.phi3d_gauss_integral(x, [sig ** 2 / 2] * 3, [0, 0, 0], nn, mm,
                                    mass=(math.pi * sig ** 2) ** 1.5)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_closed_forms_agree_2d():
    rng = np.random.default_rng(1)
    x = rng.uniform(-4, 4, (30, 2))
    setup = json.load(open(GOLDEN))["tab:2d_exmp"]["setup"]
    sig = math.sqrt(setup["sigma2"])
    n, m = np.array(setup["n"]), np.array(setup["m"])
    a = cf.phi2d_bessel(x, sig, n, m)
    b = cf.phi2d_gauss_integral(x, [sig ** 2 / 2] * 2, [0, 0], n, m, mass=math.pi * sig ** 2)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_ddi_vs_closed_form_3d_same_axis():
    # Example exmp_3d, n = m = z, sigma = 1.4, L = 8.  With R = pi/h the only error left once
    # the angular rule resolves e^{ik.x} is the spectral truncation ~ exp(-sigma^2 R^2 / 4):
    # h = 1: R = pi, h = 1/2: R = 2 pi.  The error must fall by orders of magnitude.
    errs = {}
    for h, sizes in ((1.0, (16, 32, 64)), (0.5, (32, 64, 128))):
        N = int(round(16 / h))
        n, lo, ln, X, Y, Z = _grid3(N, 8.0)
        t = qd.plan_tables(3, n, ln, (0, 0, 1), nr=sizes[0], ntheta=sizes[1], nphi=sizes[2])
        rho = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 1.4 ** 2)
        phi = nudft.ddi(rho, t, n, lo, ln)
        ex = _phi3_exact(X, Y, Z, 1.4, np.array([0, 0, 1.0]))
        errs[h] = np.linalg.norm(phi - ex) / np.linalg.norm(ex)     # Eq. error_l2
    trunc = {h: math.exp(-1.4 ** 2 * (math.pi / h) ** 2 / 4) for h in errs}
    assert errs[1.0] < 20 * trunc[1.0] and errs[0.5] < 20 * trunc[0.5], errs
    assert errs[0.5] < 1e-4 * errs[1.0]
    # the truncation really is the error left: the error is of its size, not far below it
    assert errs[1.0] > 0.05 * trunc[1.0] and errs[0.5] > 0.05 * trunc[0.5], errs


def test_ddi_vs_closed_form_2d_paper_table():
    # Example 2d_exmp / Table tab:2d_exmp, L = 8: our polar rule (2N x 2N, R = pi/h)
    # reproduces the paper's h = 1/4 accuracy level (4.7e-14) and spectral decay in h.
    setup = json.load(open(GOLDEN))["tab:2d_exmp"]
    sig = math.sqrt(setup["setup"]["sigma2"])
    nvec, mvec = np.array(setup["setup"]["n"]), np.array(setup["setup"]["m"])
    errs = {}
    for h in (0.5, 0.25):
        N = int(round(16 / h))
        n = (N, N)
        lo = (-8.0, -8.0)
        ln = (16.0, 16.0)
        t = qd.plan_tables(2, n, ln, nvec, mvec)
        ax = nudft.grid_axes(n, lo, ln)
        Y, X = np.meshgrid(ax[1], ax[0], indexing="ij")
        rho = np.exp(-(X ** 2 + Y ** 2) / sig ** 2)
        phi = nudft.ddi(rho, t, n, lo, ln)
        pts = np.stack([X.ravel(), Y.ravel()], axis=1)
        ex = cf.phi2d_bessel(pts, sig, nvec, mvec)
        r = np.linalg.norm(pts, axis=1)
        small = r < 0.1
        if small.any():
            ex[small] = cf.phi2d_gauss_integral(pts[small], [sig ** 2 / 2] * 2, [0, 0], nvec, mvec,
                                                mass=math.pi * sig ** 2)
        ex = ex.reshape(X.shape)
        errs[h] = np.linalg.norm(phi - ex) / np.linalg.norm(ex)
    assert errs[0.25] < 10 * setup["L8"]["h=1/4"], errs
    assert errs[0.5] < 1e-3 and errs[0.25] < 1e-6 * errs[0.5]


def test_ddi_vs_integral_form_anisotropic():
    # The 24^3 anisotropic Gaussian on [-6, 6)^3 with the 16 x 16 x 32 rule: the oracle's own
    # discretisation error against the derived integral form is recorded (truncation at
    # R = 2 pi leaves exp(-s_x^2 R^2 / 2) ~ 5e-5 of rhohat) and must shrink with resolution.
    from paper_1504_02897_gb300 import synth
    errs = []
    for N, sizes in ((24, (16, 16, 32)), (36, (24, 24, 48))):
        w = synth.anisotropic_gaussian_density(N, 6.0)
        n, lo, ln = w["n"], w["lo"], w["len"]
        t = qd.plan_tables(3, n, ln, (0, 0, 1), nr=sizes[0], ntheta=sizes[1], nphi=sizes[2])
        phi = nudft.ddi(w["rho"], t, n, lo, ln)
        ax = nudft.grid_axes(n, lo, ln)
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        sel = (X ** 2 + Y ** 2 + Z ** 2) <= 9.0
        pts = np.stack([X[sel], Y[sel], Z[sel]], axis=1)
        ex = cf.phi3d_gauss_integral(pts, w["s2"], [0, 0, 0], np.array([0, 0, 1.0]), mass=w["mass"])
        errs.append(np.max(np.abs(phi[sel] - ex)) / np.max(np.abs(ex)))
    assert errs[0] < 1e-3 and errs[1] < 0.1 * errs[0], errs

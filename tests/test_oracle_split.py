"""Pins of the split algorithm's oracle (Sec. 2.1, Eq. 3.9; ``oracle/split.py``): the
partition of unity itself, the smoothness of p at k = 0, the trace identity, agreement with
the paper's Erf closed form up to the predicted spectral truncation, independence of the
window width k0 and of the padding, and agreement with the spherical-quadrature oracle."""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import nudft
from oracle import quadrature as qd
from oracle import split

BALL = dict(nr=48, ntheta=32, nphi=64)


def _grid(N, L):
    n = (N, N, N)
    lo = (-L, -L, -L)
    ln = (2 * L,) * 3
    ax = [lo[d] + np.arange(N) * (2 * L / N) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return n, lo, ln, X, Y, Z


def _erf_exact(X, Y, Z, sigma, nax):
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    ex = cf.phi3d_erf(pts, sigma, nax)
    r = np.linalg.norm(pts, axis=1)
    small = r < 0.1          # the Erf form cancels catastrophically near r = 0
    if small.any():
        ex[small] = cf.phi3d_gauss_integral(pts[small], [sigma ** 2 / 2] * 3, [0, 0, 0], nax, None,
                                            mass=(math.pi * sigma ** 2) ** 1.5)
    return ex.reshape(X.shape)


def test_partition_of_unity_and_smooth_part():
    rng = np.random.default_rng(3)
    k = rng.normal(size=(200, 3)) * 2.0
    n = np.array([0.3, -0.4, 0.866]); n /= np.linalg.norm(n)
    m = np.array([0.6, 0.0, 0.8])
    k0 = 1.1
    k2 = np.sum(k * k, axis=1)
    uhat = 3 * (k @ n) * (k @ m) / k2 - n @ m
    p = split.smooth_symbol(k[:, 0], k[:, 1], k[:, 2], n, m, k0)
    assert np.max(np.abs(p + split.window(k2, k0) * uhat - uhat)) <= 1e-14
    # p is smooth at 0: along any direction p(t khat) ~ t^2 (3 (n.khat)(m.khat) - n.m) / k0^2
    khat = k[:5] / np.sqrt(k2[:5])[:, None]
    for t in (1e-3, 1e-5):
        kt = t * khat
        pt = split.smooth_symbol(kt[:, 0], kt[:, 1], kt[:, 2], n, m, k0)
        lim = t * t * (3 * (khat @ n) * (khat @ m) - n @ m) / k0 ** 2
        assert np.max(np.abs(pt - lim)) <= 1e-6 * t * t
    assert split.smooth_symbol(np.zeros(1), np.zeros(1), np.zeros(1), n, m, k0)[0] == 0.0


def test_trace_identity():
    # sum over n = e_x, e_y, e_z of the symbol is zero, in both parts
    n, lo, ln, X, Y, Z = _grid(16, 5.0)
    rho = np.exp(-(X ** 2 + 2 * Y ** 2 + Z ** 2) / 2) * (1 + 0.2 * np.sin(X + 0.3 * Z))
    s = sum(split.ddi_split(rho, n, lo, ln, e, k0=1.0, nr=12, ntheta=8, nphi=16) for e in np.eye(3))
    assert np.max(np.abs(s)) <= 1e-14 * np.max(np.abs(rho))


def test_split_matches_erf_closed_form():
    # isotropic Gaussian rho = exp(-|x|^2 / sigma^2), sigma = 1.4, n = z (Eqs.
    # extDensGausDipolar, Hessian_Ex1) on [-8, 8)^3, h = 1/2: the only error left is the
    # truncation of rhohat at the grid's band, exp(-sigma^2 (pi/h)^2 / 4) = 4e-9 of rhohat(0)
    n, lo, ln, X, Y, Z = _grid(32, 8.0)
    sigma, nax = 1.4, np.array([0.0, 0.0, 1.0])
    rho = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / sigma ** 2)
    ex = _erf_exact(X, Y, Z, sigma, nax)
    got = split.ddi_split(rho, n, lo, ln, nax, k0=0.8, **BALL)
    bound = math.exp(-sigma ** 2 * (math.pi / 0.5) ** 2 / 4)
    assert np.max(np.abs(got - ex)) / np.max(np.abs(ex)) <= bound


def test_split_two_axes_matches_erf_closed_form():
    # the axes n != m of Table tab:diff:dip (Eq. dipmn) with the Erf form of the same Gaussian:
    # p carries 3 (n.k)(m.k) - (n.m)|k|^2 and the ball weights the two-axis symbol, so an axis
    # used twice or a dropped n.m term in either part fails this
    import json
    import os
    golden = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")
    tab = json.load(open(golden))["tab:diff:dip"]["setup"]
    nax = np.array(tab["n"], float) / np.linalg.norm(tab["n"])
    m_axis = np.array(tab["m"], float) / np.linalg.norm(tab["m"])
    n, lo, ln, X, Y, Z = _grid(32, 8.0)
    sigma = 1.4
    rho = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / sigma ** 2)
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    ex = cf.phi3d_erf(pts, sigma, nax, m_axis)
    small = np.linalg.norm(pts, axis=1) < 0.1
    ex[small] = cf.phi3d_gauss_integral(pts[small], [sigma ** 2 / 2] * 3, [0, 0, 0], nax, m_axis,
                                        mass=(math.pi * sigma ** 2) ** 1.5)
    ex = ex.reshape(X.shape)
    got = split.ddi_split(rho, n, lo, ln, nax, m_axis, k0=0.8, **BALL)
    bound = math.exp(-sigma ** 2 * (math.pi / 0.5) ** 2 / 4)
    assert np.max(np.abs(got - ex)) / np.max(np.abs(ex)) <= bound


def test_window_width_does_not_matter():
    # the split is exact in the continuum: moving the window (and the ball with it) changes
    # only quadrature errors, which these rules keep at roundoff
    n, lo, ln, X, Y, Z = _grid(32, 8.0)
    rho = np.exp(-(X ** 2 / 1.5 + Y ** 2 + (Z - 0.5) ** 2 / 2.0))
    nax = np.array([math.sin(0.4), 0.0, math.cos(0.4)])
    a = split.ddi_split(rho, n, lo, ln, nax, k0=0.8, **BALL)
    b = split.ddi_split(rho, n, lo, ln, nax, k0=1.2, nr=64, ntheta=40, nphi=80)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_padding_does_not_matter():
    # p is smooth at k = 0, so its kernel decays like a Gaussian of width ~1/k0 and a 2x
    # zero padding already separates the periodic images; shown on I1 with a density whose
    # spectrum is below roundoff at the grid's band (h = 1/4: exp(-2.4 (4 pi)^2 / 4) = 1e-41)
    # so that the two k-samplings are both converged
    n, lo, ln, X, Y, Z = _grid(64, 8.0)
    rho = np.exp(-(X ** 2 / 2.4 + Y ** 2 / 2.8 + (Z - 0.5) ** 2 / 3.0))
    nax = np.array([math.sin(0.4), 0.0, math.cos(0.4)])
    a = split.split_i1(rho, n, lo, ln, nax, k0=0.8, pad=2)
    c = split.split_i1(rho, n, lo, ln, nax, k0=0.8, pad=3)
    assert np.max(np.abs(a - c)) <= 1e-10 * np.max(np.abs(a))


def test_split_agrees_with_spherical_oracle_where_both_resolve():
    # on the inner part of a resolved grid both discretisations reach the same integral
    n, lo, ln, X, Y, Z = _grid(48, 8.0)
    rho = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / 1.96)
    nax = np.array([0.0, 0.0, 1.0])
    a = split.ddi_split(rho, n, lo, ln, nax, k0=0.8, **BALL)
    b = nudft.ddi(rho, qd.plan_tables(3, n, ln, nax), n, lo, ln)
    inner = (np.abs(X) <= 3) & (np.abs(Y) <= 3) & (np.abs(Z) <= 3)
    assert np.max(np.abs(a - b)[inner]) <= 1e-10 * np.max(np.abs(a))


def test_split_operator_is_symmetric():
    # <a, Phi(b)> = <Phi(a), b> for real a, b: p is real and even in k (so the padded circular
    # convolution's kernel is symmetric) and the ball's node set is closed under k -> -k; the
    # adjoint of the time-splitting step relies on it
    rng = np.random.default_rng(5)
    n, lo, ln, X, Y, Z = _grid(16, 5.0)
    nax = np.array([0.3, -0.4, 0.866]) / np.linalg.norm([0.3, -0.4, 0.866])
    m_axis = np.array([0.6, 0.0, 0.8])
    a = rng.standard_normal(X.shape)
    b = rng.standard_normal(X.shape)
    pa = split.ddi_split(a, n, lo, ln, nax, m_axis, k0=1.0, nr=12, ntheta=8, nphi=16)
    pb = split.ddi_split(b, n, lo, ln, nax, m_axis, k0=1.0, nr=12, ntheta=8, nphi=16)
    lhs, rhs = float(np.sum(a * pb)), float(np.sum(pa * b))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), np.sum(np.abs(a * pb)))

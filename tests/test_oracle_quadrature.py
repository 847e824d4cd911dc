"""Pins of the oracle's Fourier quadrature (Sec. 2.1, Eq. DDI-Trun1) against mathematics.

Each test checks a property that an error in the rule (a wrong node, weight, Jacobian,
symbol or scale) would break, independently of the oracle's own arithmetic.
"""
import math

import numpy as np
import pytest

from oracle import quadrature as qd


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 64, 128])
def test_gauss_legendre_exactness(n):
    # n-point Gauss-Legendre integrates x^p exactly for p <= 2n-1.
    x, w = qd.gauss_legendre(n)
    assert np.all(np.diff(x) > 0)
    for p in range(0, 2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        got = float(np.sum(w * x ** p))
        assert abs(got - exact) <= 1e-14 * max(1.0, n / 8), (n, p, got, exact)


@pytest.mark.parametrize("n", [2, 5, 16, 64, 127, 256])
def test_gauss_legendre_matches_library(n):
    # Cross-check with numpy's independent implementation (eigenvalue based).
    x, w = qd.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) <= 4e-15
    # numpy scales its weights after an eigen-solve: absolute agreement is the meaningful bar
    assert np.max(np.abs(w - wr)) <= 1e-14


def test_gauss_legendre_symmetry_bitwise():
    x, w = qd.gauss_legendre(32)
    assert np.array_equal(x, -x[::-1])
    assert np.array_equal(w, w[::-1])
    x, w = qd.gauss_legendre(9)
    assert x[4] == 0.0


def _tables3(n=(16, 16, 16), length=(8.0, 8.0, 8.0), axis=(0.0, 0.0, 1.0), m=None, **kw):
    return qd.plan_tables(3, n, length, axis, m, **kw)


def test_ball_volume_and_symbol_mean():
    # sum_q w_r w_u w_phi |k|^2 = |B_R| = 4 pi R^3 / 3 (GL exact for r^2), and the symbol
    # 3 (n.khat)^2 - 1 has zero mean over the sphere, so sum W_q = 0 (Eq. DipKer).
    t = _tables3(nr=8, ntheta=6, nphi=12)
    R = t["R"]
    sym_free = qd.plan_tables(3, (16, 16, 16), (8.0, 8.0, 8.0), (0, 0, 1), (0, 0, 1), nr=8, ntheta=6, nphi=12)
    W = sym_free["W"]
    assert abs(np.sum(W)) <= 1e-14 * np.sum(np.abs(W))
    # Undo the symbol: for n = m = z, U = 3 u^2 - 1 with u = kz/|k|.
    k = t["k"]
    kn = np.linalg.norm(k, axis=1)
    U = 3 * (k[:, 2] / kn) ** 2 - 1
    mask = np.abs(U) > 1e-3
    vol = np.sum(t["W"][mask] / U[mask] * (2 * math.pi) ** 3)
    # the masked-out nodes are absent only if none are near the magic angle
    assert mask.all()
    assert abs(vol - 4 * math.pi * R ** 3 / 3) <= 1e-13 * R ** 3


def test_disk_weights_2d():
    # 2D: Jacobian |k| times |k| x symbol gives 1.5 r^2 (n_perp.khat)^2 for n = (1, 0, 0):
    # sum_q W_q (2 pi)^2 = 1.5 int_0^R r^2 dr int_0^{2pi} cos^2 = 1.5 (R^3/3) pi (GL and the
    # trapezoid are exact for these integrands).
    t = qd.plan_tables(2, (32, 32), (8.0, 8.0), (1.0, 0.0, 0.0), nr=10, nphi=16)
    total = np.sum(t["W"]) * (2 * math.pi) ** 2
    exact = 0.5 * math.pi * t["R"] ** 3
    assert abs(total - exact) <= 1e-13 * exact
    # out-of-plane axis: n = (0, 0, 1) gives -1.5 r^2, sum = -1.5 (R^3/3) 2 pi
    t = qd.plan_tables(2, (32, 32), (8.0, 8.0), (0.0, 0.0, 1.0), nr=10, nphi=16)
    total = np.sum(t["W"]) * (2 * math.pi) ** 2
    exact = -math.pi * t["R"] ** 3
    assert abs(total - exact) <= 1e-13 * abs(exact)


def test_antipodal_symmetry_bitwise():
    # The second half of the azimuth is the exact negation of the first, so every node
    # k has its partner -k with the same weight: the discrete operator is real symmetric.
    nr, nt, nph = 6, 5, 10
    t = _tables3(axis=(0.5, 0.0, math.sqrt(3) / 2), nr=nr, ntheta=nt, nphi=nph)
    k = t["k"].reshape(nr, nt, nph, 3)
    W = t["W"].reshape(nr, nt, nph)
    half = nph // 2
    for j in range(nt):
        assert np.array_equal(k[:, nt - 1 - j, half:, :], -k[:, j, :half, :])
        assert np.array_equal(W[:, nt - 1 - j, half:], W[:, j, :half])


def test_trace_of_symbol_vanishes():
    # sum_d (e_d . khat)^2 = 1 at every node, so the three axis weights sum to zero.
    kw = dict(nr=5, ntheta=4, nphi=8)
    Ws = [_tables3(axis=e, **kw)["W"] for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    tot = Ws[0] + Ws[1] + Ws[2]
    assert np.max(np.abs(tot)) <= 1e-15 * np.max(np.abs(Ws[2])) * 8


def test_two_axis_symbol_is_symmetric_part():
    # Eq. dipmn: U_nm(k) = 3 (n.khat)(m.khat) - n.m; it is symmetric in (n, m) and equals
    # the average of the single-axis symbols' polarisation identity.
    kw = dict(nr=4, ntheta=4, nphi=8)
    n = np.array([0.82778, 0.41505, -0.37751]); n /= np.linalg.norm(n)
    m = np.array([0.31180, 0.93780, -0.15214]); m /= np.linalg.norm(m)
    a = _tables3(axis=n, m=m, **kw)["W"]
    b = _tables3(axis=m, m=n, **kw)["W"]
    assert np.max(np.abs(a - b)) <= 1e-15 * np.max(np.abs(a)) * 4
    p = n + m
    q = n - m
    wp = _tables3(axis=p, m=p, **kw)["W"]
    wq = _tables3(axis=q, m=q, **kw)["W"]
    assert np.max(np.abs((wp - wq) / 4 - a)) <= 1e-14 * np.max(np.abs(a))


def test_default_kmax_and_sizes():
    t = qd.plan_tables(3, (24, 24, 24), (12.0, 12.0, 12.0), (0, 0, 1), nr=16, ntheta=16, nphi=32)
    assert t["k"].shape == (16 * 16 * 32, 3)
    assert t["R"] == math.pi / 0.5
    assert np.max(np.linalg.norm(t["k"], axis=1)) < t["R"]
    assert qd.default_sizes(3, (128, 128, 128)) == (128, 64, 128)
    assert qd.default_sizes(2, (256, 256)) == (512, 1, 512)


def test_fine_grid_start():
    k = np.array([[0.0, 1.0, -1.0], [3.0, -3.1, 0.25]])
    h = [0.5, 0.5, 0.5]
    nf = [32, 32, 32]
    l0 = qd.fine_grid_start(k, h, nf, 7)
    s = k * (0.5 * 32 / (2 * math.pi))
    assert np.all(l0 >= s - 3.5) and np.all(l0 < s - 2.5)

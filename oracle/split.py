"""The improved split algorithm of Sec. 2.1 (Eq. 3.9), 3D, written out plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

A partition of unity splits the Fourier integral of Phi = U_dip * rho:

    Phi = (2 pi)^-3 int_Omega e^{ik.x} p(k) rhohat(k) dk  +  (2 pi)^-3 int_B e^{ik.x} q(k) Uhat(k) rhohat(k) dk
        = I1 + I2,                 p = (1 - q) Uhat,

with Omega the cube |k_d| <= pi / h_d (the grid's band) and B a small ball around k = 0.
The paper requires q to be C^infinity with fast decay and p smooth; it gives no q.  Reading
used here: q(k) = exp(-|k|^2 / k0^2).  Then

    p(k) = (1 - e^{-|k|^2/k0^2}) / |k|^2 * (3 (n.k)(m.k) - (n.m) |k|^2)

is smooth at k = 0 ((1 - e^{-s})/s is entire and the bracket is a quadratic polynomial), so
its kernel in x decays faster than any power and I1 is a linear convolution evaluated with a
zero-padded FFT (the trapezoid rule in k on the padded grid's modes, spacing pi / L_d for a
2x padding).  I2 has a Gaussian-damped integrand: on the ball |k| <= c k0 (c = 6: e^{-36})
the spherical rule of ``quadrature.plan_tables`` with O(1) nodes, weights multiplied by q,
evaluated by the direct sum of ``nudft``.  rhohat is, as everywhere in the oracle, the
trapezoid sum h^3 sum_j rho_j e^{-ik.x_j}.
"""
import numpy as np

from . import nudft
from . import quadrature as qd


def window(k2, k0):
    """q(k) = exp(-|k|^2 / k0^2) as a function of |k|^2."""
    return np.exp(-k2 / (k0 * k0))


def smooth_symbol(kx, ky, kz, axis_n, axis_m, k0):
    """p(k) = (1 - q(k)) Uhat(k), Uhat = 3 (n.khat)(m.khat) - n.m, with its limit p(0) = 0."""
    n = np.asarray(axis_n, dtype=np.float64)
    m = n if axis_m is None else np.asarray(axis_m, dtype=np.float64)
    k2 = kx * kx + ky * ky + kz * kz
    nk = n[0] * kx + n[1] * ky + n[2] * kz
    mk = m[0] * kx + m[1] * ky + m[2] * kz
    poly = 3.0 * nk * mk - float(n @ m) * k2
    with np.errstate(divide="ignore", invalid="ignore"):
        f = -np.expm1(-k2 / (k0 * k0)) / k2
    f = np.where(k2 > 0, f, 1.0 / (k0 * k0))
    return f * poly


def split_i1(rho, n, lo, length, axis_n, axis_m=None, k0=1.0, pad=2):
    """I1 by the zero-padded FFT: the density sits in the first n_d points of a pad * n_d
    grid (spacing h_d); modes k = 2 pi j / (pad L_d); the result is cropped back."""
    n = tuple(int(v) for v in n)
    h = [length[d] / n[d] for d in range(3)]
    big = tuple(pad * v for v in reversed(n))              # (z, y, x)
    buf = np.zeros(big)
    buf[: n[2], : n[1], : n[0]] = rho
    kz, ky, kx = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(pad * n[d], d=h[d]) for d in (2, 1, 0)], indexing="ij")
    P = smooth_symbol(kx, ky, kz, axis_n, axis_m, k0)
    out = np.fft.ifftn(P * np.fft.fftn(buf))
    return out[: n[2], : n[1], : n[0]].real


def ball_tables(n, length, axis_n, axis_m=None, k0=1.0, ball=6.0, nr=24, ntheta=16, nphi=32):
    """Spherical rule on |k| <= ball * k0 with weights W_q q(k_q) (antipodally closed)."""
    t = qd.plan_tables(3, n, length, axis_n, axis_m, nr=nr, ntheta=ntheta, nphi=nphi, kmax=ball * k0)
    k2 = np.sum(t["k"] * t["k"], axis=1)
    return {"k": t["k"], "W": t["W"] * window(k2, k0)}


def split_i2(rho, n, lo, length, axis_n, axis_m=None, k0=1.0, **ball):
    return nudft.ddi(rho, ball_tables(n, length, axis_n, axis_m, k0, **ball), n, lo, length)


def ddi_split(rho, n, lo, length, axis_n, axis_m=None, k0=1.0, pad=2, **ball):
    """Phi = I1 + I2 (Eq. 3.9)."""
    return (split_i1(rho, n, lo, length, axis_n, axis_m, k0, pad)
            + split_i2(rho, n, lo, length, axis_n, axis_m, k0, **ball))

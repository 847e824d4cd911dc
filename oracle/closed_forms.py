"""Closed-form and 1-D-integral dipolar potentials of Gaussian densities.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``phi3d_erf``: Example exmp_3d, Eqs. extDensGausDipolar / Hessian_Ex1, for
  rho = exp(-|x|^2/sigma^2) and axes n, m:  Phi = -(n.m) rho - 3 n^T G(x) m.
* ``phi2d_bessel``: Example 2d_exmp (the I_0 / I_1 form) for rho = exp(-|x|^2/sigma^2).
* ``phi3d_gauss_integral`` / ``phi2d_gauss_integral``: for an axis-aligned anisotropic
  Gaussian rho = mass * prod_d (2 pi s_d^2)^{-1/2} exp(-(x_d-c_d)^2 / (2 s_d^2)), derived
  from the symbol the same way Sec. 2.2 derives its anisotropic references (a 1-D
  integral of Gaussian derivatives):
    3D: 1/|k|^2 = int_0^inf exp(-tau |k|^2) dtau, a_d = s_d^2 + 2 tau,
        g_tau = mass prod_d (2 pi a_d)^{-1/2} exp(-x_d^2/(2 a_d)),
        Phi = -(n.m) rho - 3 int_0^inf d_n d_m g_tau dtau,
        d_n d_m g = g [ (sum n_d x_d/a_d)(sum m_d x_d/a_d) - sum n_d m_d / a_d ].
    2D: 1/|k| = (2/sqrt(pi)) int_0^inf exp(-s^2 |k|^2) ds, a_d = s_d^2 + 2 s^2,
        Phi = -(3/sqrt(pi)) int_0^inf [ d_{n_perp m_perp} g_s - n3 m3 Lap g_s ] ds.
  The integrals are taken with scipy's adaptive quadrature after the map
  t = u / (1 - u) of [0, inf) onto [0, 1).
"""
import math

import numpy as np
from scipy import integrate, special


def _as_points(x):
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    return x


def phi3d_erf(x, sigma, n, m=None):
    """Eq. extDensGausDipolar with G from Eq. Hessian_Ex1 (rho = exp(-|x|^2/sigma^2))."""
    if m is None:
        m = n
    x = _as_points(x)
    n = np.asarray(n, float)
    m = np.asarray(m, float)
    r2 = np.sum(x * x, axis=1)
    r = np.sqrt(r2)
    rho = np.exp(-r2 / sigma ** 2)
    e = np.exp(-r2 / sigma ** 2)
    erf = special.erf(r / sigma)
    sp = math.sqrt(math.pi)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = sigma ** 2 / (2 * r2) * e - sigma ** 3 * sp / (4 * r ** 3) * erf
        b = -3 * sigma ** 2 / (2 * r2 ** 2) * e - e / r2 + 3 * sigma ** 3 * sp / (4 * r ** 5) * erf
    xn = x @ n
    xm = x @ m
    nGm = a * float(n @ m) + b * xn * xm
    return -float(n @ m) * rho - 3.0 * nGm


def phi2d_bessel(x, sigma, n, m=None):
    """Example 2d_exmp: closed form with modified Bessel functions (rho = exp(-|x|^2/sigma^2)).

    ``n``, ``m`` are 3-vectors: (n1, n2) = n_perp and n3 the out-of-plane part.
    Uses the exponentially scaled i0e/i1e for e^{-r} I_k(r).
    """
    if m is None:
        m = n
    x = _as_points(x)
    npp = np.asarray(n[:2], float)
    mpp = np.asarray(m[:2], float)
    n3, m3 = float(n[2]), float(m[2])
    r = np.sum(x * x, axis=1) / (2 * sigma ** 2)
    i0 = special.i0e(r)
    i1 = special.i1e(r)
    sp = math.sqrt(math.pi)
    xn = x @ npp
    xm = x @ mpp
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (3 * sp / (4 * sigma)) * (float(npp @ mpp) * (i0 - i1)
                                       - 2 * xn * xm / sigma ** 2 * (i0 - (1 + 2 * r) / (2 * r) * i1))
        t2 = (3 * sp * n3 * m3 * r / sigma) * (i0 - i1 - i0 / (2 * r))
    return t1 + t2


def gaussian_density(x, s2, center, mass=1.0):
    """mass * prod_d (2 pi s_d^2)^{-1/2} exp(-(x_d - c_d)^2 / (2 s_d^2)) at points x (P x d)."""
    x = _as_points(x) - np.asarray(center, float)
    s2 = np.asarray(s2, float)
    norm = mass / np.prod(np.sqrt(2 * math.pi * s2))
    return norm * np.exp(-np.sum(x * x / (2 * s2), axis=1))


def _integral(fun, rtol):
    val, _ = integrate.quad_vec(fun, 0.0, 1.0, epsabs=0.0, epsrel=rtol, limit=2000)
    return val


def phi3d_gauss_integral(x, s2, center, n, m=None, mass=1.0, rtol=1e-13):
    """Phi of an axis-aligned anisotropic 3D Gaussian by the 1-D tau integral."""
    if m is None:
        m = n
    x = _as_points(x) - np.asarray(center, float)
    s2 = np.asarray(s2, float)
    n = np.asarray(n, float)
    m = np.asarray(m, float)

    def integrand(u):
        if u >= 1.0:
            return np.zeros(x.shape[0])
        tau = u / (1.0 - u)
        jac = 1.0 / (1.0 - u) ** 2
        a = s2 + 2.0 * tau
        g = mass / np.prod(np.sqrt(2 * math.pi * a)) * np.exp(-np.sum(x * x / (2 * a), axis=1))
        xa = x / a
        val = g * ((xa @ n) * (xa @ m) - float(np.sum(n * m / a)))
        return val * jac

    rho = gaussian_density(x, s2, np.zeros(3), mass)
    return -float(n @ m) * rho - 3.0 * _integral(integrand, rtol)


def phi2d_gauss_integral(x, s2, center, n, m=None, mass=1.0, rtol=1e-13):
    """Phi of an axis-aligned anisotropic 2D Gaussian by the 1-D s integral (n, m 3-vectors)."""
    if m is None:
        m = n
    x = _as_points(x) - np.asarray(center, float)
    s2 = np.asarray(s2, float)
    npp = np.asarray(n[:2], float)
    mpp = np.asarray(m[:2], float)
    n3m3 = float(n[2]) * float(m[2])

    def integrand(u):
        if u >= 1.0:
            return np.zeros(x.shape[0])
        s = u / (1.0 - u)
        jac = 1.0 / (1.0 - u) ** 2
        a = s2 + 2.0 * s * s
        g = mass / np.prod(np.sqrt(2 * math.pi * a)) * np.exp(-np.sum(x * x / (2 * a), axis=1))
        xa = x / a
        dnm = g * ((xa @ npp) * (xa @ mpp) - float(np.sum(npp * mpp / a)))
        lap = g * (np.sum(xa * xa, axis=1) - float(np.sum(1.0 / a)))
        return (dnm - n3m3 * lap) * jac

    return -(3.0 / math.sqrt(math.pi)) * _integral(integrand, rtol)


def phi_mixture_integral(x, comps, n, m=None, dim=3, rtol=1e-13):
    """Sum of the integral forms over Gaussian components [(amp_mass, s2, center), ...]."""
    f = phi3d_gauss_integral if dim == 3 else phi2d_gauss_integral
    out = 0.0
    for mass, s2, c in comps:
        out = out + f(x, s2, c, n, m, mass=mass, rtol=rtol)
    return out

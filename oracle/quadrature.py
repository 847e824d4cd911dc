"""Fourier-space quadrature of the truncated DDI integral (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.1, Eq. DDI-Trun1: the DDI is the Fourier integral of the symbol times the
density transform over the ball |k| <= R, written in spherical (3D) or polar (2D)
coordinates so that the Jacobian |k|^{d-1} cancels the k = 0 singularity of the
symbol (Eq. DipKer; two axes n, m: Eq. dipmn).  The paper only says "high order
quadratures"; the rule used here (the same rule the CUDA library builds) is:

* radial: n_r-point Gauss-Legendre on [0, R];
* polar (3D): n_theta-point Gauss-Legendre in u = cos(theta) on [-1, 1]
  (sin(theta) d(theta) = du, so the Jacobian |k|^2 sin(theta) becomes |k|^2);
* azimuth: n_phi-point trapezoid phi_m = 2 pi m / n_phi (n_phi even); the
  second half of the azimuthal nodes is the exact negation of the first half,
  so the node set is closed under k -> -k bit for bit;
* R = k_max = pi / min_d h_d unless given.

Heterogeneous boxes (h_d unequal, e.g. the thin domains D_eps of Sec. 2.1 with
h_z = eps h_x): ``ellipsoid=True`` maps the same rule onto the ellipsoid with semi-axes
a_d = R e_d, e_d = min h / h_d (a_d = pi / h_d by default), i.e. k = e * (r khat_ball).
The Jacobian is e_x e_y (e_z); the symbol is evaluated at the direction of k,
g / |g| with g = e * khat_ball; in 2D the symbol's factor |k| is r |g|.  With equal h_d
the rule is the spherical one up to the rounding of |g| = 1.  Default polar (3D) or
azimuthal (2D) size grows with max h / min h, because the symbol at the direction of k
turns over an angular band of width ~ min e / max e of the unit sphere.

Weights of the discrete sum (so that Phi_j = Re sum_q W_q e^{i k_q.x_j} rhohat_q):
    3D: W_q = w_r w_u w_phi |k|^2 [3 (n.khat)(m.khat) - n.m] / (2 pi)^3
    2D: W_q = w_r w_phi |k| * 3[(n_perp.k)(m_perp.k) - n3 m3 |k|^2] / (2|k|) / (2 pi)^2
            = w_r w_phi 1.5 |k|^2 [(n_perp.khat)(m_perp.khat) - n3 m3] / (2 pi)^2

Every floating-point expression below is written in a fixed evaluation order with
only +, -, *, /, sqrt after the libm cos/sin calls, so that the C++ plan builder,
which follows the same order with -ffp-contract=off, produces bit-identical tables.
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def gauss_legendre(n):
    """Gauss-Legendre nodes (ascending) and weights on [-1, 1].

    Newton's method on the three-term Legendre recurrence from the initial guess
    cos(pi (i + 3/4) / (n + 1/2)) for the i-th largest root, stopped when the
    Newton update is exactly zero or after 100 updates; weight
    2 / ((1 - x^2) P_n'(x)^2).  Upper-half roots are mirrored (x -> -x, same
    weight); for odd n the middle node is exactly 0.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    half = (n + 1) // 2
    z = np.array([math.cos(math.pi * (i + 0.75) / (n + 0.5)) for i in range(half)],
                 dtype=np.float64)
    if n % 2 == 1:
        z[half - 1] = 0.0
    active = np.ones(half, dtype=bool)
    if n % 2 == 1:
        active[half - 1] = False          # the middle root is exactly zero
    iters = np.zeros(half, dtype=np.int64)

    def legendre(zz):
        p0 = np.ones_like(zz)
        p1 = zz.copy()
        for k in range(1, n):
            p0, p1 = p1, ((2 * k + 1) * zz * p1 - k * p0) / (k + 1)
        dp = n * (zz * p1 - p0) / (zz * zz - 1.0)
        return p1, dp

    while active.any():
        idx = np.nonzero(active)[0]
        zz = z[idx]
        p, dp = legendre(zz)
        dz = p / dp
        z[idx] = zz - dz
        iters[idx] += 1
        done = (dz == 0.0) | (iters[idx] >= 100)
        active[idx[done]] = False

    _, dp = legendre(z)
    w = 2.0 / ((1.0 - z * z) * dp * dp)
    x = np.empty(n)
    wt = np.empty(n)
    for i in range(half):
        x[n - 1 - i] = z[i]
        x[i] = -z[i]
        wt[n - 1 - i] = w[i]
        wt[i] = w[i]
    return x, wt


def default_sizes(dim, n, ratio=None):
    """Default quadrature sizes: (N, N/2, N) in 3D and (2N, -, 2N) in 2D (N = max grid size).
    ratio = max h / min h of an ellipsoidal rule: the 3D polar size becomes ceil(N/2 ratio),
    the 2D azimuthal size 2 ceil(N ratio)."""
    nmax = max(n[:dim])
    if dim == 3:
        if ratio is not None:
            return nmax, int(math.ceil(0.5 * nmax * ratio)), nmax
        return nmax, nmax // 2, nmax
    if ratio is not None:
        return 2 * nmax, 1, 2 * int(math.ceil(nmax * ratio))
    return 2 * nmax, 1, 2 * nmax


def azimuth_table(nphi):
    """cos/sin of the trapezoid azimuth; the second half is the exact negation of the first."""
    if nphi % 2:
        raise ValueError("n_phi must be even")
    half = nphi // 2
    c = np.empty(nphi)
    s = np.empty(nphi)
    for m in range(half):
        ang = (TWO_PI * m) / nphi
        c[m] = math.cos(ang)
        s[m] = math.sin(ang)
    c[half:] = -c[:half]
    s[half:] = -s[:half]
    return c, s


def plan_tables(dim, n, length, axis_n, axis_m=None, nr=0, ntheta=0, nphi=0, kmax=0.0, ellipsoid=False):
    """Quadrature nodes k_q (M x dim) and DDI weights W_q (M,) in node order.

    Node order: q = (i_r * n_theta + j_u) * n_phi + m in 3D, q = i_r * n_phi + m in 2D.
    ``n``/``length``: grid sizes and box lengths per axis; h_d = length_d / n_d.
    ``ellipsoid``: the rule mapped onto the ellipsoid with semi-axes R min h / h_d.
    """
    if axis_m is None:
        axis_m = axis_n
    h = [length[d] / n[d] for d in range(dim)]
    hmin = min(h)
    dnr, dnt, dnp = default_sizes(dim, n, max(h) / hmin if ellipsoid else None)
    nr = nr or dnr
    ntheta = ntheta or dnt
    nphi = nphi or dnp
    if ellipsoid:
        return _ellipsoid_tables(dim, h, hmin, axis_n, axis_m, nr, ntheta, nphi, kmax)
    if not kmax:
        kmax = math.pi / min(h)
    R = float(kmax)
    xr, wr0 = gauss_legendre(nr)
    half_R = 0.5 * R
    r = half_R * (1.0 + xr)
    wr = half_R * wr0
    c, s = azimuth_table(nphi)
    wphi = TWO_PI / nphi
    n0, n1, n2 = (float(v) for v in axis_n)
    m0, m1, m2 = (float(v) for v in axis_m)
    if dim == 3:
        u, wu = gauss_legendre(ntheta)
        st = np.sqrt((1.0 - u) * (1.0 + u))
        R3 = r[:, None, None]
        ST = st[None, :, None]
        U = u[None, :, None]
        C = c[None, None, :]
        S = s[None, None, :]
        rst = R3 * ST
        kx = rst * C
        ky = rst * S
        kz = np.broadcast_to(R3 * U, kx.shape)
        hx = ST * C
        hy = ST * S
        hz = np.broadcast_to(U, hx.shape)
        nk = (n0 * hx + n1 * hy) + n2 * hz
        mk = (m0 * hx + m1 * hy) + m2 * hz
        nm = (n0 * m0 + n1 * m1) + n2 * m2
        sym = 3.0 * (nk * mk) - nm
        tp3 = (TWO_PI * TWO_PI) * TWO_PI
        wgt = ((wr[:, None, None] * wu[None, :, None]) * wphi) * (R3 * R3)
        W = (wgt * sym) / tp3
        k = np.stack([kx.ravel(), ky.ravel(), np.ascontiguousarray(kz).ravel()], axis=1)
        return {"k": k, "W": np.ascontiguousarray(W).ravel(), "R": R,
                "sizes": (nr, ntheta, nphi), "h": h}
    R2 = r[:, None]
    C = c[None, :]
    S = s[None, :]
    kx = R2 * C
    ky = R2 * S
    nk = n0 * C + n1 * S
    mk = m0 * C + m1 * S
    sym = 1.5 * (nk * mk - n2 * m2)
    tp2 = TWO_PI * TWO_PI
    wgt = (wr[:, None] * wphi) * (R2 * R2)
    W = (wgt * sym) / tp2
    k = np.stack([kx.ravel(), ky.ravel()], axis=1)
    return {"k": k, "W": np.ascontiguousarray(W).ravel(), "R": R,
            "sizes": (nr, 1, nphi), "h": h}


def _ellipsoid_tables(dim, h, hmin, axis_n, axis_m, nr, ntheta, nphi, kmax):
    """The rule of ``plan_tables`` on the ellipsoid |k_d| <= R e_d, e_d = min h / h_d: nodes
    e * (r khat), weight w_r (w_u) w_phi r^2 (e_x e_y e_z) Uhat(g / |g|) / (2 pi)^3 in 3D and
    w_r w_phi r^2 (e_x e_y) |g| * 1.5 [(n_perp.ghat)(m_perp.ghat) - n3 m3] / (2 pi)^2 in 2D,
    g = e * khat; written as loops in the order the library evaluates them."""
    R = float(kmax) if kmax else math.pi / hmin
    e = [hmin / h[d] for d in range(dim)]
    xr, wr0 = gauss_legendre(nr)
    half_R = 0.5 * R
    r = [half_R * (1.0 + x) for x in xr]
    wr = [half_R * w for w in wr0]
    c, s = azimuth_table(nphi)
    wphi = TWO_PI / nphi
    n0, n1, n2 = (float(v) for v in axis_n)
    m0, m1, m2 = (float(v) for v in axis_m)
    if dim == 3:
        u, wu = gauss_legendre(ntheta)
        st = [math.sqrt((1.0 - v) * (1.0 + v)) for v in u]
        J = (e[0] * e[1]) * e[2]
        nm = (n0 * m0 + n1 * m1) + n2 * m2
        tp3 = (TWO_PI * TWO_PI) * TWO_PI
        M = nr * ntheta * nphi
        k = np.empty((M, 3))
        W = np.empty(M)
        q = 0
        for i in range(nr):
            for j in range(ntheta):
                rst = r[i] * st[j]
                wgt = (((wr[i] * wu[j]) * wphi) * (r[i] * r[i])) * J
                for mm in range(nphi):
                    k[q, 0] = (rst * c[mm]) * e[0]
                    k[q, 1] = (rst * s[mm]) * e[1]
                    k[q, 2] = (r[i] * u[j]) * e[2]
                    gx = (st[j] * c[mm]) * e[0]
                    gy = (st[j] * s[mm]) * e[1]
                    gz = u[j] * e[2]
                    gn = math.sqrt((gx * gx + gy * gy) + gz * gz)
                    hx, hy, hz = gx / gn, gy / gn, gz / gn
                    nk = (n0 * hx + n1 * hy) + n2 * hz
                    mk = (m0 * hx + m1 * hy) + m2 * hz
                    W[q] = (wgt * (3.0 * (nk * mk) - nm)) / tp3
                    q += 1
        return {"k": k, "W": W, "R": R, "sizes": (nr, ntheta, nphi), "h": h, "e": e}
    J = e[0] * e[1]
    tp2 = TWO_PI * TWO_PI
    M = nr * nphi
    k = np.empty((M, 2))
    W = np.empty(M)
    q = 0
    for i in range(nr):
        w0 = ((wr[i] * wphi) * (r[i] * r[i])) * J
        for mm in range(nphi):
            k[q, 0] = (r[i] * c[mm]) * e[0]
            k[q, 1] = (r[i] * s[mm]) * e[1]
            gx = c[mm] * e[0]
            gy = s[mm] * e[1]
            gn = math.sqrt(gx * gx + gy * gy)
            hx, hy = gx / gn, gy / gn
            nk = n0 * hx + n1 * hy
            mk = m0 * hx + m1 * hy
            W[q] = ((w0 * gn) * (1.5 * (nk * mk - n2 * m2))) / tp2
            q += 1
    return {"k": k, "W": W, "R": R, "sizes": (nr, 1, nphi), "h": h, "e": e}


def fine_grid_start(k, h, nf, width):
    """First fine-grid index touched by a width-w kernel centred at each node.

    The node's position on an nf-point oversampled grid (in cells, origin at the
    centre index) is s = k_d * (h_d * nf_d / (2 pi)); the first tap is
    ceil(s - w/2).  Returned as int64 (un-wrapped; the library wraps mod nf).
    """
    k = np.asarray(k)
    out = np.empty(k.shape, dtype=np.int64)
    for d in range(k.shape[1]):
        scale = (h[d] * nf[d]) / TWO_PI
        out[:, d] = np.ceil(k[:, d] * scale - 0.5 * width).astype(np.int64)
    return out

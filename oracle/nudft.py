"""The DDI as the discrete quadrature sum, evaluated by a direct nonuniform DFT.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. DDI-Con gives Phi = (2 pi)^{-d} int Uhat(k) rhohat(k) e^{i k.x} dk; Eq. DDI-Trun1
truncates it to the ball B_R in spherical/polar coordinates and Sec. 2.1 discretises
it by a quadrature.  Only grid values of rho exist, so rhohat is the trapezoid sum
h_1..h_d sum_j rho_j e^{-i k.x_j}.  The oracle evaluates exactly that sum:

    rhohat_q = h^d sum_j rho_j exp(-i k_q . x_j)                 (type 2, grid -> nodes)
    c_q      = W_q rhohat_q                                      (symbol x weights)
    Phi_j    = Re sum_q c_q exp(+i k_q . x_j)                    (type 1, nodes -> grid)

with x_j = lo + j h (j = 0..N_d-1, the duplicate periodic endpoint of Sec. 4.1 dropped).
The sums are blocked over nodes and contracted axis by axis (numpy matmul), which is
the same sum in a different association, plus a loop-level version for tiny grids.
Grid arrays are C-ordered [z][y][x] (3D) or [y][x] (2D): the last axis is x.
"""
import numpy as np


def grid_axes(n, lo, length):
    """1-D coordinate arrays x_d = lo_d + j h_d, j = 0..n_d-1, in (x, y[, z]) order."""
    return [lo[d] + np.arange(n[d]) * (length[d] / n[d]) for d in range(len(n))]


def _phases(kcol, xs, sign):
    return np.exp((sign * 1j) * np.outer(kcol, xs))


def type2(rho, k, n, lo, length, block=256):
    """rhohat_q = h^d sum_j rho_j e^{-i k_q.x_j} for every node (complex128, shape (M,))."""
    dim = len(n)
    rho = np.asarray(rho, dtype=np.float64)
    axes = grid_axes(n, lo, length)
    hprod = float(np.prod([length[d] / n[d] for d in range(dim)]))
    M = k.shape[0]
    out = np.empty(M, dtype=np.complex128)
    if dim == 3:
        nz, ny, nx = rho.shape
        flat = rho.reshape(nz * ny, nx)
        for q0 in range(0, M, block):
            kb = k[q0:q0 + block]
            ex = _phases(kb[:, 0], axes[0], -1.0)          # (Q, nx)
            ey = _phases(kb[:, 1], axes[1], -1.0)          # (Q, ny)
            ez = _phases(kb[:, 2], axes[2], -1.0)          # (Q, nz)
            t1 = (ex @ flat.T).reshape(len(kb), nz, ny)    # sum over x
            t2 = np.einsum("qzy,qy->qz", t1, ey)           # sum over y
            out[q0:q0 + block] = np.einsum("qz,qz->q", t2, ez)
    else:
        ny, nx = rho.shape
        for q0 in range(0, M, block):
            kb = k[q0:q0 + block]
            ex = _phases(kb[:, 0], axes[0], -1.0)
            ey = _phases(kb[:, 1], axes[1], -1.0)
            t1 = ex @ rho.T                                  # (Q, ny)
            out[q0:q0 + block] = np.einsum("qy,qy->q", t1, ey)
    return hprod * out


def type1(c, k, n, lo, length, block=256):
    """Phi_j = Re sum_q c_q e^{+i k_q.x_j} on the whole grid (float64, grid shape)."""
    dim = len(n)
    axes = grid_axes(n, lo, length)
    M = k.shape[0]
    if dim == 3:
        nx, ny, nz = n
        acc = np.zeros((nz, ny, nx), dtype=np.complex128)
        for q0 in range(0, M, block):
            kb = k[q0:q0 + block]
            cb = c[q0:q0 + block]
            ex = _phases(kb[:, 0], axes[0], 1.0)
            ey = _phases(kb[:, 1], axes[1], 1.0)
            ez = _phases(kb[:, 2], axes[2], 1.0) * cb[:, None]
            t = np.einsum("qz,qy->zyq", ez, ey).reshape(nz * ny, len(kb))
            acc += (t @ ex).reshape(nz, ny, nx)
    else:
        nx, ny = n
        acc = np.zeros((ny, nx), dtype=np.complex128)
        for q0 in range(0, M, block):
            kb = k[q0:q0 + block]
            cb = c[q0:q0 + block]
            ex = _phases(kb[:, 0], axes[0], 1.0)
            ey = _phases(kb[:, 1], axes[1], 1.0) * cb[:, None]
            acc += ey.T @ ex
    return acc.real


def type1_at(c, k, points, block=4096):
    """Phi at arbitrary points (P x dim): Re sum_q c_q e^{+i k_q.x_p}."""
    points = np.asarray(points, dtype=np.float64)
    out = np.zeros(points.shape[0])
    for q0 in range(0, k.shape[0], block):
        kb = k[q0:q0 + block]
        ph = np.exp(1j * (points @ kb.T))                  # (P, Q)
        out += (ph @ c[q0:q0 + block]).real
    return out


def ddi(rho, tables, n, lo, length):
    """Phi on the grid for density rho with plan tables from ``quadrature.plan_tables``."""
    k, W = tables["k"], tables["W"]
    rh = type2(rho, k, n, lo, length)
    return type1(W * rh, k, n, lo, length)


def ddi_at(rho, tables, n, lo, length, index):
    """Phi at a subset of grid points given by integer index tuples (P x dim, (x, y[, z]) order)."""
    k, W = tables["k"], tables["W"]
    rh = type2(rho, k, n, lo, length)
    index = np.asarray(index)
    pts = np.stack([lo[d] + index[:, d] * (length[d] / n[d]) for d in range(len(n))], axis=1)
    return type1_at(W * rh, k, pts)


def ddi_bruteforce(rho, tables, n, lo, length):
    """Loop-level evaluation of the same sum (tiny grids only): every term written out."""
    k, W = tables["k"], tables["W"]
    dim = len(n)
    h = [length[d] / n[d] for d in range(dim)]
    hprod = 1.0
    for v in h:
        hprod *= v
    pts = []
    vals = []
    for idx in np.ndindex(*rho.shape):
        x = [lo[d] + idx[dim - 1 - d] * h[d] for d in range(dim)]   # idx is (z, y, x)
        pts.append(x)
        vals.append(rho[idx])
    pts = np.array(pts)
    vals = np.array(vals)
    M = k.shape[0]
    rhohat = np.zeros(M, dtype=np.complex128)
    for q in range(M):
        acc = 0j
        for j in range(len(vals)):
            acc += vals[j] * np.exp(-1j * float(np.dot(k[q], pts[j])))
        rhohat[q] = hprod * acc
    phi = np.zeros(len(vals))
    for j in range(len(vals)):
        acc = 0j
        for q in range(M):
            acc += W[q] * rhohat[q] * np.exp(1j * float(np.dot(k[q], pts[j])))
        phi[j] = acc.real
    return phi.reshape(rho.shape)

"""GPE pieces around the DDI: TSFP step, energies, gradient flow, TSFP adjoint.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

All arrays are C-ordered [z][y][x] (3D) or [y][x] (2D), complex128 for psi.  The box is
periodic with N_d points per axis (Sec. 4.1, duplicate endpoint dropped); the Fourier
modes are mu_p = 2 pi p / len_d, p = -N/2..N/2-1 (numpy FFT order).  ``ddi`` is a
callable rho -> Phi (the quadrature sum of ``oracle.nudft``, or a closure over it).
"""
import numpy as np


class Grid:
    """Uniform periodic grid: sizes n = (nx, ny[, nz]), box [lo, lo + length)."""

    def __init__(self, n, lo, length):
        self.n = tuple(int(v) for v in n)
        self.lo = tuple(float(v) for v in lo)
        self.length = tuple(float(v) for v in length)
        self.dim = len(self.n)
        self.h = tuple(self.length[d] / self.n[d] for d in range(self.dim))
        self.dv = float(np.prod(self.h))
        self.shape = tuple(reversed(self.n))

    def coords(self):
        """Coordinate arrays broadcast to the grid shape, in (x, y[, z]) order."""
        axes = [self.lo[d] + np.arange(self.n[d]) * self.h[d] for d in range(self.dim)]
        mesh = np.meshgrid(*reversed(axes), indexing="ij")      # (z, y, x) order
        return list(reversed(mesh))

    def mu2(self):
        """|mu|^2 on the FFT grid (Sec. 4.1: mu_p = 2 pi p / (R - L))."""
        ks = [2 * np.pi * np.fft.fftfreq(self.n[d], d=self.h[d]) for d in range(self.dim)]
        mesh = np.meshgrid(*reversed(ks), indexing="ij")
        return sum(k * k for k in mesh)


def mass(grid, psi):
    """Discrete mass h^d sum |psi|^2 (Eq. norm)."""
    return grid.dv * float(np.sum(np.abs(psi) ** 2))


def kinetic_half(grid, psi, dt, sign=-1.0):
    """psi <- F^{-1} exp(sign * i dt |mu|^2 / 4) F psi  (first/last line of Eq. tssp2)."""
    ax = tuple(range(grid.dim))
    return np.fft.ifftn(np.exp(sign * 1j * dt * grid.mu2() / 4.0) * np.fft.fftn(psi, axes=ax), axes=ax)


def tsfp_step(grid, psi, V, beta, lam, dt, ddi):
    """One Strang step of Eq. tssp2, Case I (f = 0, sigma = 1, fixed dipole axis).

    psi1 = K psi; psi2 = psi1 exp(-i [dt V + beta dt |psi1|^2 + lam dt Phi(|psi1|^2)]);
    psi_new = K psi2, with K the half kinetic step exp(-i dt |mu|^2 / 4) in Fourier space.
    """
    psi1 = kinetic_half(grid, psi, dt)
    rho = np.abs(psi1) ** 2
    theta = V + beta * rho + lam * ddi(rho)
    psi2 = psi1 * np.exp(-1j * dt * theta)
    return kinetic_half(grid, psi2, dt)


# ---- general nonlinearity and damping (Sec. 5, Eqs. DipGPE1, tssp2, fun1, fun2) ----------
#
# i psi_t = [-1/2 Lap + V + beta |psi|^(2 sigma) + lambda Phi - i f(|psi|^2)] psi with
#   Case I   f = 0
#   Case II  f = delta                  (linear damping)
#   Case III f = delta rho^q            (q = 1: two-body, q = 2: three-body loss)
# and a fixed dipole axis.  On the nonlinear sub-step |psi|^2 = h(phi, tau) obeys
# d h / d tau = -2 f(h) h, and the sub-step is exact:
#   psi2 = psi1 exp(-i [dt V + H(phi, dt) + G(phi)]) exp(-F(phi, dt)),  phi = |psi1|^2,
#   H = beta int_0^dt h^sigma,  F = int_0^dt f(h),  G = lambda U_dip * (int_0^dt h).

def damped_density(phi, tau, damping, delta, q):
    """h(phi, tau): the density after time tau of d h / d tau = -2 f(h) h."""
    if damping == 0:
        return phi
    if damping == 1:
        return phi * np.exp(-2.0 * delta * tau)
    return phi / (1.0 + 2.0 * q * delta * tau * phi ** q) ** (1.0 / q)


def step_integrals(phi, dt, beta, sigma, damping, delta=0.0, q=1.0):
    """(H, F, g) of the nonlinear sub-step in closed form (the paper's Cases I-III), with
    g = int_0^dt h(phi, tau) d tau, so that G = lambda U_dip * g."""
    phi = np.asarray(phi, dtype=np.float64)
    if damping == 0:
        return beta * phi ** sigma * dt, np.zeros_like(phi), phi * dt
    if damping == 1:
        H = beta * phi ** sigma / (2.0 * delta * sigma) * (-np.expm1(-2.0 * delta * sigma * dt))
        F = np.full_like(phi, delta * dt)
        g = phi / (2.0 * delta) * (-np.expm1(-2.0 * delta * dt))
        return H, F, g
    x = 2.0 * q * delta * dt * phi ** q        # 1 + x = (phi / h(phi, dt))^q
    L = np.log1p(x)
    F = L / (2.0 * q)
    if sigma == q:
        H = beta / (2.0 * q * delta) * L
    else:
        H = beta * phi ** (sigma - q) / (2.0 * delta * (q - sigma)) * np.expm1((1.0 - sigma / q) * L)
    if q == 1:
        g = np.log1p(2.0 * delta * dt * phi) / (2.0 * delta)
    else:
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.expm1((1.0 - 1.0 / q) * L) / (2.0 * delta * (q - 1.0) * phi ** (q - 1.0))
        g = np.where(phi > 0, g, 0.0)
    return H, F, g


def tsfp_step_general(grid, psi, V, beta, lam, dt, ddi, sigma=1.0, damping=0, delta=0.0, q=1.0):
    """One Strang step of Eq. tssp2 for Eq. DipGPE1 with a fixed dipole axis."""
    psi1 = kinetic_half(grid, psi, dt)
    phi = np.abs(psi1) ** 2
    H, F, g = step_integrals(phi, dt, beta, sigma, damping, delta, q)
    theta = dt * V + H + lam * ddi(g)
    psi2 = psi1 * np.exp(-1j * theta) * np.exp(-F)
    return kinetic_half(grid, psi2, dt)


def tsfp_run_general(grid, psi, coeffs, t0, dt, nsteps, ddi, sigma=1.0, damping=0, delta=0.0, q=1.0):
    """Strang steps with time-dependent V, beta, lambda (Sec. 5, e.g. Example dy_app_damp):
    coeffs(t) -> (V, beta, lambda), frozen over each step at its midpoint t0 + (k + 1/2) dt,
    which keeps the splitting second order where the coefficients are smooth in t."""
    for k in range(nsteps):
        V, beta, lam = coeffs(t0 + (k + 0.5) * dt)
        psi = tsfp_step_general(grid, psi, V, beta, lam, dt, ddi, sigma, damping, delta, q)
    return psi


def energies(grid, phi, V, beta, lam, ddi):
    """Energy split of Sec. 3.2: E_kin, E_pot, E_int, E_dip, E, mu, virial I, mass."""
    ax = tuple(range(grid.dim))
    phihat = np.fft.fftn(phi, axes=ax)
    ntot = phi.size
    ekin = 0.5 * grid.dv / ntot * float(np.sum(grid.mu2() * np.abs(phihat) ** 2))
    rho = np.abs(phi) ** 2
    epot = grid.dv * float(np.sum(V * rho))
    eint = 0.5 * beta * grid.dv * float(np.sum(rho * rho))
    edip = 0.5 * lam * grid.dv * float(np.sum(ddi(rho) * rho)) if lam != 0.0 else 0.0
    e = ekin + epot + eint + edip
    return {"E": e, "mu": e + eint + edip, "Ekin": ekin, "Epot": epot, "Eint": eint,
            "Edip": edip, "virial": 2 * ekin - 2 * epot + 3 * eint + 3 * edip,
            "mass": grid.dv * float(np.sum(rho))}


def gf_step(grid, phi, V, beta, lam, dt, ddi, inner_tol=1e-13, inner_max=200):
    """One backward-Euler step of the normalised gradient flow (Eqs. gf-eq2..gffg33).

    The paper omits how the implicit equation
        (phi1 - phi) / dt = [1/2 Lap - V - beta |phi|^2 - lam Phi] phi1
    is solved.  Reading used here: the stabilised fixed point with
        W = V + beta |phi|^2 + lam Phi(|phi|^2),  alpha = (max W + min W) / 2,
        phi1^(m+1) = F^{-1}[ F(phi/dt + (alpha - W) phi1^(m)) / (1/dt + alpha + |mu|^2/2) ],
    started from phi1^(0) = phi, stopped when max |phi1^(m+1) - phi1^(m)| <= inner_tol or
    after inner_max sweeps; then phi_new = phi1 / sqrt(h^d sum |phi1|^2).
    Returns (phi_new, inner_iterations).
    """
    ax = tuple(range(grid.dim))
    rho = np.abs(phi) ** 2
    W = V + beta * rho + (lam * ddi(rho) if lam != 0.0 else 0.0)
    alpha = 0.5 * (float(W.max()) + float(W.min()))
    denom = 1.0 / dt + alpha + 0.5 * grid.mu2()
    rhs0 = phi / dt
    cur = phi
    it = 0
    for it in range(1, inner_max + 1):
        nxt = np.fft.ifftn(np.fft.fftn(rhs0 + (alpha - W) * cur, axes=ax) / denom, axes=ax)
        diff = float(np.max(np.abs(nxt - cur)))
        cur = nxt
        if diff <= inner_tol:
            break
    nrm = np.sqrt(mass(grid, cur))
    return cur / nrm, it


def ground_state(grid, phi0, V, beta, lam, dt, ddi, tol=1e-10, max_steps=100000,
                 rule="energy", inner_tol=1e-13):
    """Iterate ``gf_step`` from phi0 (normalised first).

    rule "energy": stop when |E^{n+1} - E^n| < tol; rule "paper": stop when
    max |phi^{n+1} - phi^n| / dt <= tol (Sec. 3.2).  Returns (phi, steps, energies list).
    """
    phi = phi0 / np.sqrt(mass(grid, phi0))
    hist = [energies(grid, phi, V, beta, lam, ddi)["E"]]
    for n in range(1, max_steps + 1):
        new, _ = gf_step(grid, phi, V, beta, lam, dt, ddi, inner_tol=inner_tol)
        e = energies(grid, new, V, beta, lam, ddi)["E"]
        hist.append(e)
        if rule == "energy":
            done = abs(e - hist[-2]) < tol
        else:
            done = float(np.max(np.abs(new - phi))) / dt <= tol
        phi = new
        if done:
            return phi, n, hist
    return phi, max_steps, hist


def tsfp_forward(grid, psi0, V, beta, lam, dt, nsteps, ddi):
    """Run nsteps of ``tsfp_step``; returns the final psi."""
    psi = psi0
    for _ in range(nsteps):
        psi = tsfp_step(grid, psi, V, beta, lam, dt, ddi)
    return psi


def observable_z2(grid, psi):
    """J = h^d sum z^2 |psi|^2 (the final-time <z^2>), 3D; uses y in 2D."""
    c = grid.coords()
    z = c[-1]
    return grid.dv * float(np.sum(z * z * np.abs(psi) ** 2))


def tsfp_tangent(grid, psi0, V, beta, lam, dt, nsteps, ddi, dpsi0, dV):
    """Tangent-linear model of ``nsteps`` TSFP steps: the first-order change of psi_T for a
    change dpsi0 of psi0 and dV of the trap (same in every step).  One step, with
    psi1 = K psi, rho = |psi1|^2, theta = V + beta rho + lam A rho, psi2 = psi1 exp(-i dt theta):
        dpsi1 = K dpsi,  drho = 2 Re(conj(psi1) dpsi1),  dtheta = dV + beta drho + lam A drho,
        dpsi2 = dpsi1 exp(-i dt theta) - i dt dtheta psi2,  dpsi_out = K dpsi2."""
    psi, d = psi0, dpsi0
    for _ in range(nsteps):
        psi1 = kinetic_half(grid, psi, dt)
        d1 = kinetic_half(grid, d, dt)
        rho = np.abs(psi1) ** 2
        ph = np.exp(-1j * dt * (V + beta * rho + lam * ddi(rho)))
        psi2 = psi1 * ph
        drho = 2.0 * np.real(np.conj(psi1) * d1)
        dtheta = dV + beta * drho + (lam * ddi(drho) if lam != 0.0 else 0.0)
        d2 = d1 * ph - 1j * dt * dtheta * psi2
        psi = kinetic_half(grid, psi2, dt)
        d = kinetic_half(grid, d2, dt)
    return d


def tsfp_adjoint(grid, psi0, V, beta, lam, dt, nsteps, ddi, gT=None, return_cot=False):
    """Gradient dJ/dV_j (plain partial derivatives w.r.t. grid values) of J = <z^2>(psi_T).

    Pairing <a, b> = Re h^d sum conj(a) b.  For the nonlinear step
    psi2 = psi1 exp(-i dt theta), theta = V + beta |psi1|^2 + lam A|psi1|^2 (A symmetric):
        r   = Re(conj(-i dt psi2) g2)
        dJ/dV += h^d r
        g1  = exp(+i dt theta) g2 + 2 psi1 (beta r + lam A r)
    and the kinetic half step K has adjoint K* = F^{-1} exp(+i dt |mu|^2/4) F.
    Forward states are recomputed from stored step inputs (all steps stored: oracle).
    Returns (grad_V, J), and with ``return_cot`` also the cotangent of psi0.
    """
    states = [psi0]
    psi = psi0
    for _ in range(nsteps):
        psi = tsfp_step(grid, psi, V, beta, lam, dt, ddi)
        states.append(psi)
    c = grid.coords()
    z = c[-1]
    psiT = states[-1]
    J = grid.dv * float(np.sum(z * z * np.abs(psiT) ** 2))
    g = 2.0 * z * z * psiT if gT is None else gT
    grad = np.zeros(grid.shape)
    for s in range(nsteps - 1, -1, -1):
        psi_in = states[s]
        psi1 = kinetic_half(grid, psi_in, dt)
        rho = np.abs(psi1) ** 2
        theta = V + beta * rho + lam * ddi(rho)
        ph = np.exp(-1j * dt * theta)
        psi2 = psi1 * ph
        g2 = kinetic_half(grid, g, dt, sign=+1.0)
        r = np.real(np.conj(-1j * dt * psi2) * g2)
        grad += grid.dv * r
        s_field = beta * r + (lam * ddi(r) if lam != 0.0 else 0.0)
        g1 = np.conj(ph) * g2 + 2.0 * psi1 * s_field
        g = kinetic_half(grid, g1, dt, sign=+1.0)
    if return_cot:
        return grad, J, g
    return grad, J

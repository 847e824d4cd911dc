"""Pins of the oracle GPE pieces (Secs. 3-4) against invariants, exact solutions and the
paper's printed convergence rates."""
import json
import math
import os

import numpy as np
import pytest

from oracle import gpe
from oracle import nudft
from oracle import quadrature as qd
from paper_1504_02897_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _setup(N, L, axis=(0, 0, 1), sizes=(0, 0, 0)):
    n, lo, ln = synth.box(N, L)
    grid = gpe.Grid(n, lo, ln)
    t = qd.plan_tables(3, n, ln, axis, nr=sizes[0], ntheta=sizes[1], nphi=sizes[2])
    return grid, (lambda rho: nudft.ddi(rho, t, n, lo, ln)), n, lo, ln


def test_tsfp_conserves_mass():
    # Each sub-step of Eq. tssp2 is unitary on the grid (Eq. norm is conserved exactly).
    grid, ddi, n, lo, ln = _setup(12, 5.0)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 2))
    psi = synth.gpe_initial(n, lo, ln, (1, 1, 2), eps=0.05, seed=1)
    m0 = gpe.mass(grid, psi)
    for _ in range(10):
        psi = gpe.tsfp_step(grid, psi, V, 20.0, 8.0, 0.01, ddi)
    assert abs(gpe.mass(grid, psi) - m0) <= 1e-13


def test_tsfp_linear_case_is_exact_propagator():
    # beta = lam = 0, V = 0: the scheme is the exact free propagator exp(-i t |mu|^2/2).
    grid, ddi, n, lo, ln = _setup(12, 5.0)
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 1), eps=0.1, seed=2)
    psi = gpe.tsfp_forward(grid, psi0, np.zeros(grid.shape), 0.0, 0.0, 0.05, 4, ddi)
    exact = np.fft.ifftn(np.exp(-0.5j * 0.2 * grid.mu2()) * np.fft.fftn(psi0))
    assert np.max(np.abs(psi - exact)) <= 1e-13


def test_tsfp_second_order_in_time():
    # Sec. 4.2 setup (box [-8,8]^3, V=|x|^2/2, psi0 = pi^{-3/4} exp(-|x|^2/2), n=z,
    # lambda = beta/2, beta = 2, t = 0.28) on a coarse grid: halving dt divides the error
    # by 4 (the paper prints rates 2.001-2.011 in Table spatial_temporal_3d_dy).
    tab = json.load(open(GOLDEN))["spatial_temporal_3d_dy"]
    grid, ddi, n, lo, ln = _setup(16, 8.0)
    X, Y, Z = synth.coords(n, lo, ln)
    V = 0.5 * (X ** 2 + Y ** 2 + Z ** 2)
    psi0 = (math.pi ** -0.75) * np.exp(-0.5 * (X ** 2 + Y ** 2 + Z ** 2)).astype(complex)
    beta, lam, T = 2.0, 1.0, 0.28
    dt0 = tab["dt0"]
    sols = [gpe.tsfp_forward(grid, psi0, V, beta, lam, dt0 / 2 ** k, 35 * 2 ** k, ddi) for k in range(4)]
    # successive differences of a second-order scheme shrink by 4 per halving
    diffs = [np.linalg.norm(sols[k] - sols[k + 1]) for k in range(3)]
    rates = [math.log2(diffs[i] / diffs[i + 1]) for i in range(2)]
    assert all(abs(r - 2.0) < 0.05 for r in rates), (diffs, rates)
    # error of the dt0 run (Richardson: |psi(dt0) - psi(dt0/8)| * 64/63), context only:
    # the same order of magnitude as the paper's 2.983e-6 at dt = 0.008
    err0 = np.linalg.norm(sols[0] - sols[3]) / np.linalg.norm(sols[3]) * 64 / 63
    assert 0.1 * tab["beta=2"][0] < err0 < 10 * tab["beta=2"][0], err0


def test_tsfp_energy_conservation_second_order():
    grid, ddi, n, lo, ln = _setup(12, 6.0)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 1))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 1), eps=0.05, seed=3)
    e0 = gpe.energies(grid, psi0, V, 10.0, 5.0, ddi)["E"]
    drift = []
    for dt in (0.02, 0.01):
        psi = gpe.tsfp_forward(grid, psi0, V, 10.0, 5.0, dt, int(round(0.2 / dt)), ddi)
        drift.append(abs(gpe.energies(grid, psi, V, 10.0, 5.0, ddi)["E"] - e0))
    assert drift[1] < drift[0] / 3.0 and drift[0] < 1e-3, drift


def test_gradient_flow_linear_oscillator_exact():
    # beta = lam = 0: the ground state of V = (x^2 + y^2 + z^2/4)/2 has E = (1+1+1/2)/2
    # = 1.25 and E_kin = E_pot (virial with no interactions).
    n, lo, ln = (32, 32, 48), (-8.0, -8.0, -12.0), (16.0, 16.0, 24.0)
    grid = gpe.Grid(n, lo, ln)
    ddi = None                                     # lam = 0: the DDI is never called
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 0.5))
    phi0 = synth.gpe_initial(n, lo, ln, (1.3, 0.8, 0.6))
    # the paper's stopping rule (Sec. 3.2): max|phi^{n+1} - phi^n| / dt <= eps0
    phi, steps, hist = gpe.ground_state(grid, phi0, V, 0.0, 0.0, 1.0, ddi, tol=1e-10, rule="paper")
    e = gpe.energies(grid, phi, V, 0.0, 0.0, ddi)
    # E is variational (error quadratic in the state error) and lands on 1.25; the state
    # itself is only as converged as the stabilised inner solve allows at dt = 1 (whose
    # contraction is |alpha - W| / (1/dt + alpha) ~ 0.97 here), so its first-order
    # quantities carry ~1e-6: E_kin - E_pot and the distance to the exact Gaussian.
    assert abs(e["E"] - 1.25) <= 1e-11
    assert abs(e["Ekin"] - e["Epot"]) <= 1e-5
    exact = synth.gpe_initial(n, lo, ln, (1, 1, 0.5)).real
    assert np.max(np.abs(np.abs(phi) - exact)) <= 1e-5
    assert np.all(np.diff(hist) <= 1e-14)          # energy never increases


def test_gradient_flow_energy_decreases_with_ddi():
    grid, ddi, n, lo, ln = _setup(12, 6.0, axis=(0.5, 0, math.sqrt(0.75)))
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 2))
    phi = synth.gpe_initial(n, lo, ln, (1, 1, 2), eps=0.1, seed=4).real.astype(complex)
    e_prev = gpe.energies(grid, phi, V, 30.0, 12.0, ddi)["E"]
    for _ in range(15):
        phi, _ = gpe.gf_step(grid, phi, V, 30.0, 12.0, 0.01, ddi)
        e = gpe.energies(grid, phi, V, 30.0, 12.0, ddi)["E"]
        assert e <= e_prev + 1e-12
        e_prev = e
    assert abs(gpe.mass(grid, phi) - 1.0) <= 1e-13


@pytest.mark.slow
def test_virial_identity_no_ddi():
    # Sec. 3.2, Eq. vir_iden with lambda = 0 (beta = 207.16, V = (x^2+y^2+z^2/4)/2):
    # at convergence I = 2E_kin - 2E_pot + 3E_int is ~0, and E approaches the printed
    # lambda = 0 row of Table virial_dip3d (2.7943) on this coarser grid.
    tab = json.load(open(GOLDEN))["virial_dip3d"]
    row = [r for r in tab["rows"] if r[0] == 0.0][0]
    n, lo, ln = (32, 32, 40), (-8.0, -8.0, -12.0), (16.0, 16.0, 24.0)
    grid = gpe.Grid(n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 0.5))
    phi0 = synth.gpe_initial(n, lo, ln, (1, 1, 0.5))
    phi, steps, hist = gpe.ground_state(grid, phi0, V, 207.16, 0.0, 0.2, lambda r: 0 * r, tol=1e-12,
                                        inner_tol=1e-12)
    e = gpe.energies(grid, phi, V, 207.16, 0.0, lambda r: 0 * r)
    assert abs(e["virial"]) < 1e-3 * e["E"]
    assert abs(e["E"] - row[1]) < 2e-3 * row[1], e


@pytest.mark.slow
@pytest.mark.parametrize("lam,n,tol", [(103.58, (24, 24, 32), 1e-4), (-103.58, (20, 20, 24), 2e-3)])
def test_virial_table_rows_with_ddi(lam, n, tol):
    # Sec. 3.2, Table virial_dip3d, rows lambda = +-103.58 (beta = 207.16, V = (x^2+y^2+z^2/4)/2,
    # dipole axis z): the oracle's normalised gradient flow with its direct-sum DDI reaches the
    # printed E, mu, E_kin, E_pot, E_int and E_dip on grids coarser than the paper's (h = 2/3,
    # 3/4 here; at 24 x 24 x 32 every part agrees to the printed 5 digits within 1e-4), and the
    # virial I = 2E_kin - 2E_pot + 3E_int + 3E_dip (Eq. vir_iden) vanishes.  The sign and size of
    # E_dip pin the DDI's sign and scale inside the ground-state iteration.
    tab = json.load(open(GOLDEN))["virial_dip3d"]
    row = [r for r in tab["rows"] if abs(r[0] - lam) < 1e-9][0]
    lo, ln = (-8.0, -8.0, -12.0), (16.0, 16.0, 24.0)
    grid = gpe.Grid(n, lo, ln)
    t = qd.plan_tables(3, n, ln, (0, 0, 1))
    ddi = lambda r: nudft.ddi(r, t, n, lo, ln)  # noqa: E731
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 0.5))
    phi0 = synth.gpe_initial(n, lo, ln, (1, 1, 0.5))
    phi, _, _ = gpe.ground_state(grid, phi0, V, 207.16, lam, 0.2, ddi, tol=1e-10, inner_tol=1e-10)
    e = gpe.energies(grid, phi, V, 207.16, lam, ddi)
    for k, j in (("E", 1), ("mu", 2), ("Ekin", 3), ("Epot", 4), ("Eint", 5), ("Edip", 6)):
        assert abs(e[k] - row[j]) <= tol * abs(row[j]), (k, e[k], row[j])
    assert abs(e["virial"]) <= tol * e["E"], e


def test_adjoint_matches_finite_differences():
    # dJ/dV from the hand-derived adjoint vs central differences of the forward map.
    grid, ddi, n, lo, ln = _setup(10, 5.0, axis=(0.5, 0, math.sqrt(0.75)))
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 2))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 2), eps=0.05, seed=5)
    beta, lam, dt, steps = 15.0, 6.0, 0.01, 6
    grad, J = gpe.tsfp_adjoint(grid, psi0, V, beta, lam, dt, steps, ddi)
    for d in synth.trap_directions(n, count=2, seed=9):
        eps = 1e-4
        jp = gpe.observable_z2(grid, gpe.tsfp_forward(grid, psi0, V + eps * d, beta, lam, dt, steps, ddi))
        jm = gpe.observable_z2(grid, gpe.tsfp_forward(grid, psi0, V - eps * d, beta, lam, dt, steps, ddi))
        fd = (jp - jm) / (2 * eps)
        ad = float(np.sum(grad * d))
        assert abs(fd - ad) <= 1e-7 * max(abs(fd), 1e-12) + 1e-13, (fd, ad)


# ---- general nonlinearity and damping (Sec. 5): the closed forms of H, F, G -----------------

CASES = [  # (sigma, damping, delta, q): Case I cubic and quintic, Case II, Case III (sigma = q and not)
    (1.0, 0, 0.0, 1.0), (2.0, 0, 0.0, 1.0), (1.0, 1, 0.3, 1.0), (2.0, 1, 0.7, 1.0),
    (1.0, 2, 0.4, 1.0), (1.0, 2, 0.4, 2.0), (2.0, 2, 0.25, 1.0), (2.0, 2, 0.25, 2.0), (1.5, 2, 0.5, 3.0),
]


@pytest.mark.parametrize("sigma,damping,delta,q", CASES)
def test_step_integrals_match_their_definitions(sigma, damping, delta, q):
    # H = beta int_0^dt h^sigma, F = int_0^dt f(h), g = int_0^dt h with d h / d tau = -2 f(h) h
    # (Eqs. fun1, fun2): integrate that ODE system numerically and compare the closed forms
    from scipy.integrate import solve_ivp
    beta, dt = 3.0, 0.37
    f = (lambda r: 0.0 * r) if damping == 0 else ((lambda r: delta + 0.0 * r) if damping == 1 else (lambda r: delta * r ** q))
    for phi in (1e-6, 0.05, 0.8, 2.5):
        def rhs(_, y):
            h = y[0]
            return [-2.0 * f(h) * h, beta * h ** sigma, f(h), h]
        sol = solve_ivp(rhs, (0.0, dt), [phi, 0.0, 0.0, 0.0], method="DOP853", rtol=1e-13, atol=1e-16)
        h_end, H_ref, F_ref, g_ref = sol.y[:, -1]
        H, F, g = gpe.step_integrals(np.array([phi]), dt, beta, sigma, damping, delta, q)
        assert abs(H[0] - H_ref) <= 1e-10 * max(abs(H_ref), 1e-300)
        assert abs(F[0] - F_ref) <= 1e-10 * max(abs(F_ref), 1e-12)
        assert abs(g[0] - g_ref) <= 1e-10 * abs(g_ref)
        assert abs(gpe.damped_density(phi, dt, damping, delta, q) - h_end) <= 1e-10 * h_end


def _small_gpe(N=16, L=5.0):
    n, lo, ln = synth.box(N, L)
    grid = gpe.Grid(n, lo, ln)
    t = qd.plan_tables(3, n, ln, (0.0, 0.0, 1.0))
    ddi = lambda rho: nudft.ddi(rho, t, n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 2))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 2), eps=0.05, seed=7)
    return grid, ddi, V, psi0


def test_general_step_case_i_equals_tsfp_step():
    grid, ddi, V, psi0 = _small_gpe()
    a = gpe.tsfp_step(grid, psi0, V, 20.0, 8.0, 0.01, ddi)
    b = gpe.tsfp_step_general(grid, psi0, V, 20.0, 8.0, 0.01, ddi, sigma=1.0, damping=0)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_linear_damping_mass_decays_exactly():
    # Case II: dN/dt = -2 delta N (Eq. Mass_Disp) and the scheme reproduces it exactly
    grid, ddi, V, psi0 = _small_gpe()
    delta, dt = 0.2, 0.01
    psi = psi0
    m0 = gpe.mass(grid, psi)
    for k in range(1, 6):
        psi = gpe.tsfp_step_general(grid, psi, V, 20.0, 8.0, dt, ddi, sigma=1.0, damping=1, delta=delta)
        assert abs(gpe.mass(grid, psi) - m0 * math.exp(-2 * delta * k * dt)) <= 1e-12 * m0


def test_nonlinear_damping_mass_dissipation_law():
    # Case III, q = 2 (three-body loss): over one step the mass loss matches
    # 2 int_0^dt h^d sum f(h) h, i.e. the grid sum of phi - h(phi, dt), to roundoff
    grid, ddi, V, psi0 = _small_gpe()
    delta, q, dt = 0.5, 2.0, 0.02
    psi1 = gpe.kinetic_half(grid, psi0, dt)
    phi = np.abs(psi1) ** 2
    psi = gpe.tsfp_step_general(grid, psi0, V, 20.0, 8.0, dt, ddi, sigma=1.0, damping=2, delta=delta, q=q)
    loss = gpe.mass(grid, psi0) - gpe.mass(grid, psi)
    expected = grid.dv * float(np.sum(phi - gpe.damped_density(phi, dt, 2, delta, q)))
    assert abs(loss - expected) <= 1e-12 * gpe.mass(grid, psi0)


def test_damping_to_zero_recovers_case_i():
    grid, ddi, V, psi0 = _small_gpe()
    a = gpe.tsfp_step_general(grid, psi0, V, 20.0, 8.0, 0.01, ddi, sigma=1.0, damping=0)
    for damping, q in ((1, 1.0), (2, 1.0), (2, 2.0)):
        b = gpe.tsfp_step_general(grid, psi0, V, 20.0, 8.0, 0.01, ddi, sigma=1.0, damping=damping,
                                  delta=1e-9, q=q)
        assert np.max(np.abs(a - b)) <= 1e-7 * np.max(np.abs(a))


@pytest.mark.parametrize("nsteps", [1, 3])
def test_adjoint_dot_product_identity(nsteps):
    # <S' d, g> = <d_psi, S'^T g>_psi + sum_j dV_j (S'^T g)_V,j for the tangent-linear model S'
    # of the time-splitting steps and the hand-written adjoint, to roundoff (pairing
    # <a, b> = Re h^d sum conj(a) b; the V-part of the adjoint is a plain partial derivative)
    grid, ddi, V, psi0 = _small_gpe(N=12, L=4.0)
    beta, lam, dt = 20.0, 8.0, 0.02
    rng = np.random.default_rng(11)
    dpsi = rng.standard_normal(grid.shape) + 1j * rng.standard_normal(grid.shape)
    dV = rng.standard_normal(grid.shape)
    g = rng.standard_normal(grid.shape) + 1j * rng.standard_normal(grid.shape)
    dT = gpe.tsfp_tangent(grid, psi0, V, beta, lam, dt, nsteps, ddi, dpsi, dV)
    lhs = grid.dv * float(np.real(np.sum(np.conj(dT) * g)))
    gV, _, gpsi = gpe.tsfp_adjoint(grid, psi0, V, beta, lam, dt, nsteps, ddi, gT=g, return_cot=True)
    rhs = grid.dv * float(np.real(np.sum(np.conj(dpsi) * gpsi))) + float(np.sum(dV * gV))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_tangent_linear_model_matches_finite_differences():
    # the tangent-linear model against central differences of the steps themselves
    grid, ddi, V, psi0 = _small_gpe(N=12, L=4.0)
    beta, lam, dt, nsteps, eps = 20.0, 8.0, 0.02, 2, 1e-6
    rng = np.random.default_rng(12)
    dpsi = 0.1 * (rng.standard_normal(grid.shape) + 1j * rng.standard_normal(grid.shape))
    dV = 0.1 * rng.standard_normal(grid.shape)
    fwd = lambda s: gpe.tsfp_forward(grid, psi0 + s * dpsi, V + s * dV, beta, lam, dt, nsteps, ddi)
    fd = (fwd(eps) - fwd(-eps)) / (2 * eps)
    tl = gpe.tsfp_tangent(grid, psi0, V, beta, lam, dt, nsteps, ddi, dpsi, dV)
    assert np.max(np.abs(fd - tl)) <= 1e-7 * np.max(np.abs(tl))


def test_time_dependent_run_is_second_order():
    # coefficients frozen at each step's midpoint keep Strang splitting second order for smooth
    # beta(t), lambda(t) (here with three-body loss, Case III); freezing them at the step's
    # start (the same run with the schedule shifted by dt/2) is only first order
    grid, ddi, n, lo, ln = _setup(16, 8.0)
    X, Y, Z = synth.coords(n, lo, ln)
    V = 0.5 * (X ** 2 + Y ** 2 + Z ** 2)
    psi0 = (math.pi ** -0.75) * np.exp(-0.5 * (X ** 2 + Y ** 2 + Z ** 2)).astype(complex)

    def coeffs(t):
        beta = 2.0 * (1.0 + 0.5 * math.sin(10.0 * t))
        return V, beta, 0.5 * beta

    def run(dt, shift):
        return gpe.tsfp_run_general(grid, psi0, lambda t: coeffs(t - shift * dt), 0.0, dt, int(round(0.28 / dt)),
                                    ddi, 1.0, 2, 0.5, 2.0)

    for shift, order in ((0.0, 2.0), (0.5, 1.0)):
        sols = [run(0.008 / 2 ** k, shift) for k in range(3)]
        d = [np.linalg.norm(sols[k] - sols[k + 1]) for k in range(2)]
        assert abs(math.log2(d[0] / d[1]) - order) < 0.15, (shift, d)


def test_collapse_schedule_is_continuous():
    # Example dy_app_damp: b(t) and beta(t) are continuous at their breakpoints; the last
    # nonzero branch is the printed 38.8066 (see synth.collapse_schedule for the reading)
    eps = 1e-9
    assert abs(synth.collapse_b(0.4) - synth.collapse_b(0.4 + eps)) < 1e-7
    for tb in (3.2, 3.6):
        a, b = synth.collapse_schedule(tb)[1], synth.collapse_schedule(tb + eps)[1]
        assert abs(a - b) <= 1e-6 * abs(a)
    assert abs(synth.collapse_schedule(4.8)[1] - 38.8066) <= 1e-4
    assert synth.collapse_schedule(0.0)[1] == pytest.approx(761.102 * 0.9)
    assert synth.collapse_schedule(3.4)[1] == pytest.approx(761.102 * 0.3)
    assert synth.collapse_schedule(4.2)[0] and not synth.collapse_schedule(4.2 + eps)[0]
    assert synth.collapse_schedule(5.8)[2] == 82.864 and synth.collapse_schedule(5.8 + eps)[2] == 0.0
    assert synth.collapse_schedule(5.8 + eps)[1] == 0.0

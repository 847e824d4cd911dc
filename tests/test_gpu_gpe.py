"""GPU parity of the GPE layer (TSFP step, energies, gradient flow, adjoint) against the
FP64 oracle, plus the paper's printed ground-state energies (Table virial_dip3d)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import gpe as ogpe
from oracle import nudft
from oracle import quadrature as qd
from paper_1504_02897_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


@pytest.fixture(scope="module")
def D():
    from paper_1504_02897_gb300 import build, ddi
    build.build()
    ddi.load()
    return ddi


def _setup(N, L, axis=(0.5, 0.0, math.sqrt(0.75)), gam=(1, 1, 2)):
    n, lo, ln = synth.box(N, L)
    grid = ogpe.Grid(n, lo, ln)
    t = qd.plan_tables(3, n, ln, axis)
    ddi = lambda rho: nudft.ddi(rho, t, n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, gam)
    psi0 = synth.gpe_initial(n, lo, ln, gam, eps=0.05, seed=3)
    return n, lo, ln, grid, ddi, V, psi0


def _t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def _in(x, precision):
    """The state or trap as an FP32 plan receives it (the oracle then runs on that input)."""
    if precision == 0:
        return x
    return x.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(x) else x.astype(np.float32).astype(np.float64)


def _report(name, err, tol):
    print(f"[{name}] rel err {err:.3e} (tol {tol:.0e})")
    return err


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_tsfp_steps_match_oracle(D, precision, tol):
    # FP32: the oracle runs on the FP32-rounded state and trap, the inputs the path receives
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    beta, lam, dt, steps = 20.0, 8.0, 0.01, 5
    ref = ogpe.tsfp_forward(grid, _in(psi0, precision), _in(V, precision), beta, lam, dt, steps, ddi)
    plan = D.Plan(3, n, lo, ln, (0.5, 0.0, math.sqrt(0.75)), precision=precision)
    psi = _t(psi0, plan.cplx_dtype)
    plan.gpe_step(psi, _t(V, plan.real_dtype), beta, lam, dt, steps)
    got = psi.cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert _report(f"tsfp 16^3 x5 prec={precision}", err, tol) <= tol


def test_tsfp_32cubed_many_steps_error_growth(D):
    # FP64 at 32^3 with the paper's dynamics setup of Sec. 4.2 (V = |x|^2 / 2, lambda = beta / 2):
    # 1e-12 after one step, and the growth of the difference over 40 steps reported and bounded
    # (each step is unitary up to roundoff, so differences grow slowly)
    import torch
    n, lo, ln = synth.box(32, 8.0)
    axis = (0.0, 0.0, 1.0)
    grid = ogpe.Grid(n, lo, ln)
    t = qd.plan_tables(3, n, ln, axis)
    ddi = lambda rho: nudft.ddi(rho, t, n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 1))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 1), eps=0.05, seed=5)
    beta, lam, dt = 10.0, 5.0, 0.008
    plan = D.Plan(3, n, lo, ln, axis, precision=0)
    psi = _t(psi0, torch.complex128)
    Vt = _t(V, torch.float64)
    ref = psi0
    errs = []
    for k in range(40):
        ref = ogpe.tsfp_step(grid, ref, V, beta, lam, dt, ddi)
        plan.gpe_step(psi, Vt, beta, lam, dt, 1)
        if k in (0, 9, 19, 39):
            errs.append(np.max(np.abs(psi.cpu().numpy() - ref)) / np.max(np.abs(ref)))
    print("[tsfp 32^3 fp64] rel err after 1, 10, 20, 40 steps: " + ", ".join(f"{e:.2e}" for e in errs))
    assert errs[0] <= 1e-12
    assert errs[-1] <= 2e-11


def test_tsfp_128cubed_one_step(D):
    # one FP64 step at the full 128^3 size (configs 3/4's box and trap) against the oracle, whose
    # DDI is the direct quadrature sum over all 1,048,576 nodes (a few minutes on the host)
    import torch
    n, lo, ln = synth.box(128, 10.0)
    axis = (0.0, 0.0, 1.0)
    grid = ogpe.Grid(n, lo, ln)
    t = qd.plan_tables(3, n, ln, axis)
    ddi = lambda rho: nudft.ddi(rho, t, n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, (1.0, 1.0, 2.0))
    psi0 = synth.gpe_initial(n, lo, ln, (1.0, 1.0, 2.0), eps=0.05, seed=0)
    beta, lam, dt = 207.16, 0.16 * 207.16, 1e-3
    ref = ogpe.tsfp_step(grid, psi0, V, beta, lam, dt, ddi)
    plan = D.Plan(3, n, lo, ln, axis, precision=0)
    psi = _t(psi0, torch.complex128)
    plan.gpe_step(psi, _t(V, torch.float64), beta, lam, dt, 1)
    err = np.max(np.abs(psi.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert _report("tsfp 128^3 fp64, one step", err, 1e-12) <= 1e-12


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_energies_match_oracle(D, precision, tol):
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    ref = ogpe.energies(grid, _in(psi0, precision), _in(V, precision), 30.0, 12.0, ddi)
    plan = D.Plan(3, n, lo, ln, (0.5, 0.0, math.sqrt(0.75)), precision=precision)
    got = plan.gpe_energy(_t(psi0, plan.cplx_dtype), _t(V, plan.real_dtype), 30.0, 12.0)
    for key in ("E", "mu", "Ekin", "Epot", "Eint", "Edip", "mass"):
        err = abs(got[key] - ref[key]) / max(1.0, abs(ref[key]))
        _report(f"energy {key} prec={precision}", err, tol)
        assert err <= tol, (key, got[key], ref[key])


def test_tsfp_mass_conservation_fp32_64(D):
    import torch
    n, lo, ln = synth.box(64, 8.0)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 2))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 2), eps=0.05, seed=4)
    plan = D.Plan(3, n, lo, ln, (0.0, 0.0, 1.0), precision=1)
    psi = _t(psi0, torch.complex64)
    Vt = _t(V, torch.float32)
    m0 = plan.gpe_energy(psi, Vt, 0.0, 0.0)["mass"]
    plan.gpe_step(psi, Vt, 207.16, 33.1456, 1e-3, 400)
    m1 = plan.gpe_energy(psi, Vt, 0.0, 0.0)["mass"]
    # Every sub-step is unitary (Sec. 4.1).  In FP32 the twiddles are applied to FP64
    # accuracy (head + tail) and the phase factors as v + v (e - 1), so no rounded factor
    # with |w| != 1 repeats from step to step: the mass takes only the unbiased rounding
    # of each operation.  Pin: drift <= 1e-5 over 400 steps.
    assert abs(m1 - m0) <= 1e-5


def test_gradient_flow_steps_match_oracle(D):
    # max_steps = 4 with an unreachable tolerance: both sides take exactly 4 BE steps
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    phi0 = psi0.real.astype(np.complex128)
    beta, lam, dt = 30.0, 12.0, 0.01
    phi = phi0 / math.sqrt(ogpe.mass(grid, phi0))
    for _ in range(4):
        phi, _ = ogpe.gf_step(grid, phi, V, beta, lam, dt, ddi)
    plan = D.Plan(3, n, lo, ln, (0.5, 0.0, math.sqrt(0.75)), precision=0)
    g = _t(phi0, plan.cplx_dtype)
    st = plan.ground_state(g, _t(V, plan.real_dtype), beta, lam, dt, 1e-300, rule=D.STOP_PAPER, max_steps=4)
    assert not st["converged"] and st["steps"] == 4
    got = g.cpu().numpy()
    assert np.max(np.abs(got - phi)) / np.max(np.abs(phi)) <= 1e-11


def test_adjoint_matches_oracle_and_fd(D):
    import torch
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    beta, lam, dt, steps = 15.0, 6.0, 0.01, 6
    ref_grad, ref_J = ogpe.tsfp_adjoint(grid, psi0, V, beta, lam, dt, steps, ddi)
    plan = D.Plan(3, n, lo, ln, (0.5, 0.0, math.sqrt(0.75)), precision=0)
    Vt = _t(V, torch.float64)
    J, grad = D.trap_gradient(plan, _t(psi0, torch.complex128), Vt, beta, lam, dt, steps, checkpoint=4)
    assert abs(J - ref_J) <= 1e-12 * abs(ref_J)
    g = grad.cpu().numpy()
    assert np.max(np.abs(g - ref_grad)) <= 1e-10 * np.max(np.abs(ref_grad))
    # central differences of the GPU forward map
    for d in synth.trap_directions(n, count=2, seed=9):
        eps = 1e-4
        vals = []
        for sgn in (1, -1):
            psi = _t(psi0, torch.complex128)
            plan.gpe_step(psi, _t(V + sgn * eps * d, torch.float64), beta, lam, dt, steps)
            vals.append(ogpe.observable_z2(grid, psi.cpu().numpy()))
        fd = (vals[0] - vals[1]) / (2 * eps)
        ad = float(np.sum(g * d))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)


def test_trap_gradient_driver_and_autograd(D):
    # the checkpointed driver behind the C ABI: the checkpoint spacing changes only what is
    # recomputed, so the gradient is the same bits for every spacing; the autograd Function
    # runs the forward alone in forward (J as the oracle's) and the adjoint in backward
    import torch
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    beta, lam, dt, steps = 15.0, 6.0, 0.01, 6
    ref_grad, ref_J = ogpe.tsfp_adjoint(grid, psi0, V, beta, lam, dt, steps, ddi)
    plan = D.Plan(3, n, lo, ln, (0.5, 0.0, math.sqrt(0.75)), precision=0)
    Vt = _t(V, torch.float64)
    p0 = _t(psi0, torch.complex128)
    grads = []
    for ck in (1, 3, 6, 9):
        J, g = plan.trap_gradient(p0, Vt, beta, lam, dt, steps, checkpoint=ck)
        assert abs(J - ref_J) <= 1e-12 * abs(ref_J)
        grads.append(g.clone())
    for g in grads[1:]:
        assert torch.equal(g, grads[0])
    assert np.max(np.abs(grads[0].cpu().numpy() - ref_grad)) <= 1e-10 * np.max(np.abs(ref_grad))
    Jf, psiT = plan.trap_observable(p0, Vt, beta, lam, dt, steps)
    assert abs(Jf - ref_J) <= 1e-12 * abs(ref_J)
    assert torch.equal(p0, _t(psi0, torch.complex128))          # psi0 is read only
    Vg = Vt.clone().requires_grad_(True)
    out = D.TrapGradient.apply(plan, p0, Vg, beta, lam, dt, steps, checkpoint=3)
    assert abs(float(out.detach()) - ref_J) <= 1e-12 * abs(ref_J)
    (2.0 * out).backward()
    assert torch.equal(Vg.grad, 2.0 * grads[0])


def test_trap_gradient_rejects_short_workspace(D):
    import ctypes
    import torch
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    plan = D.Plan(3, n, lo, ln, (0.0, 0.0, 1.0), precision=0)
    lib = D.load()
    nbytes = ctypes.c_size_t(0)
    assert lib.gpe_trap_gradient_workspace(plan._h, 10, 4, ctypes.byref(nbytes)) == 0
    assert nbytes.value == (3 + 4 + 2) * 16 ** 3 * 16
    work = torch.empty(nbytes.value - 16, dtype=torch.uint8, device="cuda")
    J = ctypes.c_double(0.0)
    Vt = _t(V, torch.float64)
    g = torch.empty_like(Vt)
    st = lib.gpe_trap_gradient(plan._h, ctypes.c_void_p(_t(psi0, torch.complex128).data_ptr()),
                               ctypes.c_void_p(Vt.data_ptr()), 1.0, 0.0, 0.01, 10, 4, ctypes.c_void_p(work.data_ptr()),
                               nbytes.value - 16, ctypes.byref(J), ctypes.c_void_p(g.data_ptr()), None)
    assert st == -1 and b"workspace" in lib.ddi_last_error()


@pytest.mark.parametrize("row,rule", [(0, 0), (2, 0), (4, 1)])
def test_virial_table_ground_state_energies(D, row, rule):
    # Table virial_dip3d (beta = 207.16, V = (x^2+y^2+z^2/4)/2, [-12,12]^3, h = 1/4, n = z):
    # the GPU gradient flow reproduces the printed energies to their 5 significant figures.
    import torch
    tab = json.load(open(GOLDEN))["virial_dip3d"]
    lam, E, mu, Ekin, Epot, Eint, Edip, I = tab["rows"][row]
    n, lo, ln = synth.box(96, 12.0)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 0.5))
    phi0 = synth.gpe_initial(n, lo, ln, (1, 1, 0.5))
    plan = D.Plan(3, n, lo, ln, (0.0, 0.0, 1.0), precision=0)
    phi = _t(phi0, torch.complex128)
    # rule 0: |E^{n+1} - E^n| < 1e-12; rule 1: the paper's max|phi^{n+1} - phi^n| / dt <= 1e-10
    tol = 1e-12 if rule == 0 else 1e-10
    st = plan.ground_state(phi, _t(V, torch.float64), 207.16, lam, 0.01, tol, rule=rule, max_steps=40000,
                           check_every=10)
    assert st["converged"]
    for got, want in ((st["E"], E), (st["mu"], mu), (st["Ekin"], Ekin), (st["Epot"], Epot), (st["Eint"], Eint)):
        assert abs(got - want) <= 0.6 * 10 ** (math.floor(math.log10(abs(want))) - 4), (got, want)
    if Edip != 0.0:
        assert abs(st["Edip"] - Edip) <= 0.6 * 10 ** (math.floor(math.log10(abs(Edip))) - 4)
    # I is first order in the state error: ~1e-6 after the energy rule; the paper's rule
    # reaches the printed 1e-10 level (Table virial_dip3d: |I^h| <= 6.7e-10)
    assert abs(st["virial"]) <= (1e-5 if rule == 0 else 1e-8), st["virial"]


@pytest.mark.parametrize("sigma,damping,delta,q", [
    (1.0, 0, 0.0, 1.0), (2.0, 0, 0.0, 1.0), (1.0, 1, 0.3, 1.0), (1.0, 2, 0.4, 1.0), (1.0, 2, 0.4, 2.0),
    (2.0, 2, 0.25, 1.0),
])
def test_general_step_matches_oracle(D, sigma, damping, delta, q):
    # Sec. 5: cubic/quintic nonlinearity, no / linear / two- and three-body damping, FP64
    # path against the oracle's closed-form step (itself pinned against Eqs. fun1, fun2)
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    beta, lam, dt, steps = 20.0, 8.0, 0.01, 3
    ref = psi0
    for _ in range(steps):
        ref = ogpe.tsfp_step_general(grid, ref, V, beta, lam, dt, ddi, sigma, damping, delta, q)
    plan = D.Plan(3, n, lo, ln, (0.5, 0.0, math.sqrt(0.75)), precision=0)
    psi = _t(psi0, plan.cplx_dtype)
    plan.gpe_step_ex(psi, _t(V, plan.real_dtype), beta, lam, dt, steps, sigma, damping, delta, q)
    got = psi.cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-12


def test_general_step_fp32_three_body_loss(D):
    import torch
    n, lo, ln, grid, ddi, V, psi0 = _setup(16, 5.0)
    beta, lam, dt, steps = 20.0, 8.0, 0.01, 5
    ref = _in(psi0, 1)
    for _ in range(steps):
        ref = ogpe.tsfp_step_general(grid, ref, _in(V, 1), beta, lam, dt, ddi, 1.0, 2, 0.5, 2.0)
    plan = D.Plan(3, n, lo, ln, (0.5, 0.0, math.sqrt(0.75)), precision=1)
    psi = _t(psi0, torch.complex64)
    plan.gpe_step_ex(psi, _t(V, torch.float32), beta, lam, dt, steps, 1.0, D.DAMP_POWER, 0.5, 2.0)
    got = psi.cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert _report("general step fp32, three-body loss", err, 1e-6) <= 1e-6
    with pytest.raises(D.DDIError):
        plan.gpe_step_ex(psi, _t(V, torch.float32), beta, lam, dt, 1, 1.0, D.DAMP_LINEAR, 0.0)  # delta must be > 0


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_tsfp_2d_matches_oracle(D, precision, tol):
    # 2D dynamics (the paper's 2D TS-NUFFT): polar quadrature, n_perp / n_3 axis, 4 Strang steps
    n, lo, ln = synth.box(32, 6.0, 2)
    axis = (math.sin(0.6), 0.0, math.cos(0.6))
    grid = ogpe.Grid(n, lo, ln)
    t = qd.plan_tables(2, n, ln, axis)
    ddi = lambda rho: nudft.ddi(rho, t, n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, (1, 1.5))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1.5), eps=0.05, seed=2)
    beta, lam, dt, steps = 15.0, 6.0, 0.01, 4
    ref = ogpe.tsfp_forward(grid, _in(psi0, precision), _in(V, precision), beta, lam, dt, steps, ddi)
    plan = D.Plan(2, n, lo, ln, axis, precision=precision)
    psi = _t(psi0, plan.cplx_dtype)
    plan.gpe_step(psi, _t(V, plan.real_dtype), beta, lam, dt, steps)
    got = psi.cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert _report(f"tsfp 2d 32^2 x4 prec={precision}", err, tol) <= tol

"""Time-dependent coefficients on the GPU (Sec. 5, Example dy_app_damp): Plan.gpe_run steps
the general GPE with the collapse example's trap switch, beta(t) and lambda(t) and its
three-body loss (f = delta rho^2, delta = 3.512), each step one gpe_step_ex with the
coefficients at the step's midpoint, against the oracle's tsfp_run_general (FP64, 1e-12).
The segments cross the breakpoints t = 3.2 (beta), 4.2 (trap off) and 4.8 (beta)."""
import numpy as np
import pytest

from oracle import gpe as ogpe
from oracle import nudft
from oracle import quadrature as qd
from paper_1504_02897_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import torch
    from paper_1504_02897_gb300 import build, ddi
    build.build()
    ddi.load()
    torch.cuda.init()
    return ddi


def test_collapse_schedule_matches_oracle(D):
    import torch
    n, lo, ln = synth.box(16, 6.0)
    grid = ogpe.Grid(n, lo, ln)
    axis = (0.0, 0.0, 1.0)
    t = qd.plan_tables(3, n, ln, axis)

    def ddi(rho):
        return nudft.ddi(rho, t, n, lo, ln)

    V_on = synth.harmonic_trap(n, lo, ln, synth.COLLAPSE_GAMMAS)
    V_off = np.zeros_like(V_on)
    psi0 = synth.gpe_initial(n, lo, ln, synth.COLLAPSE_GAMMAS, eps=0.05, seed=9)
    damp = dict(sigma=1.0, damping=2, delta=3.512, q=2.0)

    def coeffs_np(tt):
        trap, beta, lam = synth.collapse_schedule(tt)
        return (V_on if trap else V_off), beta, lam

    plan = D.Plan(3, n, lo, ln, axis, precision=0)
    Vt_on = torch.from_numpy(V_on).cuda()
    Vt_off = torch.zeros_like(Vt_on)

    def coeffs_gpu(tt):
        trap, beta, lam = synth.collapse_schedule(tt)
        return (Vt_on if trap else Vt_off), beta, lam

    ref = psi0
    psi = torch.from_numpy(psi0).cuda()
    for t0 in (3.1, 4.1, 4.7):
        ref = ogpe.tsfp_run_general(grid, ref, coeffs_np, t0, 0.05, 4, ddi, **damp)
        plan.gpe_run(psi, coeffs_gpu, t0, 0.05, 4, **damp)
    got = psi.cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-12
    # the three-body loss removed mass (Case III dissipates)
    assert ogpe.mass(grid, ref) < ogpe.mass(grid, psi0)

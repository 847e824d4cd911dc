"""GPU parity of the improved split algorithm (Sec. 2.1, Eq. 3.9; plans with split_k0 != 0)
against the oracle's ``split.ddi_split``: the smooth part I1 by the 2x zero-padded FFT
convolution with p = (1 - q) Uhat on the fine grid's modes, and the small-ball part I2 by the
spherical rule on |k| <= 6 k0 with weights times the window q.  Tolerances as for the DDI:
1e-12 (FP64 plans) and 1e-6 (FP32 plans) of max |oracle|."""
import math

import numpy as np
import pytest

from oracle import gpe as ogpe
from oracle import nudft
from oracle import split
from paper_1504_02897_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}


@pytest.fixture(scope="module")
def D():
    import torch
    from paper_1504_02897_gb300 import build, ddi
    build.build()
    ddi.load()
    torch.cuda.init()
    return ddi


def _relinf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _case(name):
    if name == "cube64":
        # h = 1/4: the ball's taps fill about half of each fine axis, so the band skips lines
        n, lo, ln = synth.box(64, 8.0)
        X, Y, Z = synth.coords(n, lo, ln)
        rho = np.exp(-(X ** 2 / 1.5 + Y ** 2 + (Z - 0.5) ** 2 / 2.0))
        return dict(n=n, lo=lo, ln=ln, rho=rho, axis=_unit((math.sin(0.4), 0.0, math.cos(0.4))), m=None, k0=0.8,
                    sizes=dict(nr=48, ntheta=32, nphi=64))
    if name == "cube32":
        n, lo, ln = synth.box(32, 8.0)
        X, Y, Z = synth.coords(n, lo, ln)
        rho = np.exp(-(X ** 2 / 1.5 + Y ** 2 + (Z - 0.5) ** 2 / 2.0))
        return dict(n=n, lo=lo, ln=ln, rho=rho, axis=_unit((math.sin(0.4), 0.0, math.cos(0.4))), m=None, k0=0.8,
                    sizes=dict(nr=48, ntheta=32, nphi=64))
    # ragged sizes and box lengths, two different axes (Eq. dipmn)
    n, lo, ln = (32, 16, 24), (-6.0, -3.0, -5.0), (12.0, 7.0, 10.0)
    X, Y, Z = synth.coords(n, lo, ln)
    rho = np.exp(-(X ** 2 / 2 + (Y - 0.3) ** 2 + Z ** 2 / 1.5)) * (1 + 0.2 * np.sin(X + 0.5 * Z))
    return dict(n=n, lo=lo, ln=ln, rho=rho, axis=_unit((0.5, 0.0, math.sqrt(0.75))), m=_unit((0.6, 0.0, 0.8)),
                k0=1.3, sizes=dict(nr=24, ntheta=16, nphi=40))


def _plan(D, c, precision, **kw):
    # every line of the fine grid transformed (the band of lines around k = 0 that the ball's
    # taps need is compared with this at the end of the file)
    kw.setdefault("split_full_passes", True)
    return D.Plan(3, c["n"], c["lo"], c["ln"], c["axis"], c["m"], precision=precision, split_k0=c["k0"],
                  **c["sizes"], **kw)


@pytest.mark.parametrize("name", ["cube32", "ragged"])
@pytest.mark.parametrize("precision", [0, 1])
def test_split_matches_oracle(D, name, precision):
    c = _case(name)
    plan = _plan(D, c, precision)
    assert plan.info.split_k0 == c["k0"]
    got = plan.apply(_t(c["rho"], plan.real_dtype)).double().cpu().numpy()
    ref = split.ddi_split(c["rho"], c["n"], c["lo"], c["ln"], c["axis"], c["m"], k0=c["k0"], **c["sizes"])
    tol = TOL[precision]
    if precision:
        # FP32: against the oracle on the FP32-rounded density, the input the path receives
        ref = split.ddi_split(c["rho"].astype(np.float32).astype(np.float64), c["n"], c["lo"], c["ln"], c["axis"],
                              c["m"], k0=c["k0"], **c["sizes"])
    err = _relinf(got, ref)
    print(f"[split {name} prec={precision}] rel err {err:.3e} (tol {tol:.1e})")
    assert err <= tol


def test_split_parts_through_the_stages(D):
    # I2 = type-1 of the type-2 on the ball's nodes (ddi_type2 / ddi_type1 of a split plan);
    # I1 = Phi - I2; each against its oracle part, so a failure names the part
    c = _case("ragged")
    plan = _plan(D, c, 0)
    rho = _t(c["rho"], plan.real_dtype)
    phi = plan.apply(rho).cpu().numpy()
    i2 = plan.type1(plan.type2(rho)).cpu().numpy()
    ref1 = split.split_i1(c["rho"], c["n"], c["lo"], c["ln"], c["axis"], c["m"], k0=c["k0"])
    ref2 = split.split_i2(c["rho"], c["n"], c["lo"], c["ln"], c["axis"], c["m"], k0=c["k0"], **c["sizes"])
    scale = np.max(np.abs(ref1 + ref2))
    assert np.max(np.abs(i2 - ref2)) <= 1e-12 * scale
    assert np.max(np.abs((phi - i2) - ref1)) <= 1e-12 * scale


def test_split_in_place(D):
    # rho and phi may alias: the smooth part reads rho before anything writes phi
    import torch
    c = _case("cube32")
    plan = _plan(D, c, 1)
    rho = _t(c["rho"], plan.real_dtype)
    out = plan.apply(rho)
    buf = rho.clone()
    plan.apply(buf, out=buf)
    torch.cuda.synchronize()
    assert torch.equal(out, buf)


def test_split_set_axes_equals_fresh_plan(D):
    # the ball's weights are rebuilt on the device and the smooth symbol takes the new axes
    import torch
    c = _case("ragged")
    plan = _plan(D, c, 1)
    rho = _t(c["rho"], plan.real_dtype)
    plan.apply(rho)
    a1, m1 = _unit((0.3, -0.5, 0.8)), _unit((0.7, 0.1, -0.2))
    plan.set_axes(a1, m1)
    got = plan.apply(rho)
    fresh = D.Plan(3, c["n"], c["lo"], c["ln"], a1, m1, precision=1, split_k0=c["k0"], split_full_passes=True,
                   **c["sizes"])
    ref = fresh.apply(rho)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_split_time_splitting_step(D):
    # gpe_step on a split plan: the DDI of every step is Eq. 3.9's (FP64, 3 Strang steps)
    N, L = 24, 6.0
    n, lo, ln = synth.box(N, L)
    grid = ogpe.Grid(n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 2))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 2), eps=0.05, seed=8)
    axis = _unit((math.sin(0.5), 0.0, math.cos(0.5)))
    k0, sizes = 1.0, dict(nr=24, ntheta=16, nphi=32)
    beta, lam, dt, steps = 20.0, 8.0, 0.02, 3

    def ddi(rho):
        return split.ddi_split(rho, n, lo, ln, axis, None, k0=k0, **sizes)

    ref = psi0
    for _ in range(steps):
        ref = ogpe.tsfp_step(grid, ref, V, beta, lam, dt, ddi)
    plan = D.Plan(3, n, lo, ln, axis, precision=0, split_k0=k0, split_full_passes=True, **sizes)
    psi = _t(psi0, plan.cplx_dtype)
    plan.gpe_step(psi, _t(V, plan.real_dtype), beta, lam, dt, steps)
    got = psi.cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-12


def test_split_adjoint_gradient(D):
    # the split operator is symmetric (p and the ball's weights are real and even), so the
    # hand-written adjoint's Phi(r) is valid with it: trap gradient through 4 steps on a split
    # plan against the oracle's adjoint with the split DDI (FP64)
    import torch
    N, L = 24, 6.0
    n, lo, ln = synth.box(N, L)
    grid = ogpe.Grid(n, lo, ln)
    V = synth.harmonic_trap(n, lo, ln, (1, 1, 2))
    psi0 = synth.gpe_initial(n, lo, ln, (1, 1, 2), eps=0.05, seed=10)
    axis = _unit((0.5, 0.0, 0.8))
    k0, sizes = 1.0, dict(nr=24, ntheta=16, nphi=32)
    beta, lam, dt, steps = 15.0, 6.0, 0.01, 4

    def ddi(rho):
        return split.ddi_split(rho, n, lo, ln, axis, None, k0=k0, **sizes)

    ref_grad, ref_J = ogpe.tsfp_adjoint(grid, psi0, V, beta, lam, dt, steps, ddi)
    plan = D.Plan(3, n, lo, ln, axis, precision=0, split_k0=k0, split_full_passes=True, **sizes)
    J, grad = D.trap_gradient(plan, _t(psi0, torch.complex128), _t(V, torch.float64), beta, lam, dt, steps,
                              checkpoint=2)
    assert abs(J - ref_J) <= 1e-12 * abs(ref_J)
    g = grad.cpu().numpy()
    assert np.max(np.abs(g - ref_grad)) <= 1e-10 * np.max(np.abs(ref_grad))


@pytest.mark.parametrize("name", ["cube64", "cube32", "ragged"])
@pytest.mark.parametrize("precision", [0, 1])
def test_split_band_equals_full_passes(D, name, precision):
    # the lines the band skips are zero (spread) or never read (interpolation), and the FFT of
    # zeros is exactly zero, so the banded plan (the default) computes the same bits
    import torch
    c = _case(name)
    full = _plan(D, c, precision)
    band = _plan(D, c, precision, split_full_passes=False)
    rho = _t(c["rho"], full.real_dtype)
    a = full.apply(rho)
    b = band.apply(rho)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.fixture(scope="module")
def full_split_ref():
    # the 128^3 mixture workload with the library's default split parameters (k0 = 9.6 / 24,
    # ball 6 k0, 48 x 32 x 64 nodes): I1 on the whole grid by the oracle's padded FFT, and
    # rhohat at all ball nodes, from which I2 costs one ball sum per sampled point
    w = synth.gaussian_mixture_density(128, 12.0, seed=0)
    k0 = 9.6 / 24.0
    sizes = dict(nr=48, ntheta=32, nphi=64)
    i1 = split.split_i1(w["rho"], w["n"], w["lo"], w["len"], w["axis"], None, k0=k0)
    tb = split.ball_tables(w["n"], w["len"], w["axis"], None, k0=k0, **sizes)
    rh = nudft.type2(w["rho"], tb["k"], w["n"], w["lo"], w["len"], block=512)
    return w, i1, tb, rh


@pytest.mark.parametrize("precision", [0, 1])
def test_split_full_size_sampled_points(D, full_split_ref, precision):
    import torch
    w, i1, tb, rh = full_split_ref
    plan = D.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, split_k0=-1.0, tile=(-1, 0, 0))
    assert int(plan.info.nodes) == 48 * 32 * 64
    phi = plan.apply(torch.from_numpy(w["rho"]).to("cuda", plan.real_dtype)).double().cpu().numpy()
    rng = np.random.default_rng(11)
    idx = rng.integers(0, 128, size=(1000, 3))
    idx[:6] = [[64, 64, 64], [0, 0, 0], [127, 127, 127], [1, 64, 127], [127, 0, 64], [60, 70, 64]]
    pts = np.stack([w["lo"][d] + idx[:, d] * (w["len"][d] / 128) for d in range(3)], axis=1)
    ref = i1[idx[:, 2], idx[:, 1], idx[:, 0]] + nudft.type1_at(tb["W"] * rh, tb["k"], pts)
    got = phi[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert _relinf(got, ref) <= TOL[precision]


def test_describe_equals_the_built_plan(D):
    # ddi_plan_describe (host only) reports what ddi_plan_create builds
    w = synth.gaussian_mixture_density(32, 8.0, seed=1)
    for kw in (dict(precision=1), dict(precision=0, split_k0=0.8), dict(precision=1, split_k0=0.8),
               dict(precision=0, ellipsoid=True)):
        desc = D.make_desc(3, w["n"], w["lo"], w["len"], w["axis"], **kw)
        want = D.describe(desc)
        plan = D.Plan(3, w["n"], w["lo"], w["len"], w["axis"], **kw)
        got = plan.info
        for f in ("dim", "precision", "width", "nodes", "nodes_used", "nr", "ntheta", "nphi", "ellipsoid"):
            assert getattr(got, f) == getattr(want, f), f
        assert list(got.nf) == list(want.nf) and list(got.band) == list(want.band)
        assert got.kmax == want.kmax and got.split_k0 == want.split_k0
        plan.close()

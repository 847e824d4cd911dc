"""GPU parity of the DDI path (through the C ABI) against the FP64 oracle.

Tolerances (relative L-infinity, normalised by max |oracle|): 1e-12 for FP64 plans,
1e-6 for FP32 plans, whose reference is the oracle evaluated on the input rounded to
FP32 (the data the FP32 path receives), so the input's own rounding is not charged to the
path.  Every FP32 test prints the error it reached.  Full-size 128^3 checks compare the
type-2 stage on sampled nodes and the type-1 stage (on seeded random node values) at
sampled grid points, each against the oracle's per-node / per-point sums, in the plan
bench.py times."""
import math

import numpy as np
import pytest

from oracle import nudft
from oracle import quadrature as qd
from paper_1504_02897_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}


def _in(x, precision):
    """The input as the plan receives it: rounded to FP32 for FP32 plans."""
    return x.astype(np.float32).astype(np.float64) if precision == 1 else x


def _report(name, precision, err):
    print(f"[{name} prec={precision}] rel err {err:.3e} (tol {TOL[precision]:.0e})")
    return err


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


def _plan(D, dim, n, lo, ln, axis, m=None, precision=0, **kw):
    return D.Plan(dim, n, lo, ln, axis, m, precision=precision, **kw)


def _run(D, plan, rho_np):
    import torch
    rho = torch.from_numpy(np.ascontiguousarray(rho_np)).to("cuda", plan.real_dtype)
    out = plan.apply(rho)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def _oracle(rho, n, lo, ln, axis, m=None, sizes=(0, 0, 0), dim=3):
    t = qd.plan_tables(dim, n, ln, axis, m, nr=sizes[0], ntheta=sizes[1], nphi=sizes[2])
    return nudft.ddi(rho, t, n, lo, ln)


@pytest.mark.parametrize("precision", [0, 1])
def test_ddi_anisotropic_gaussian_24(D, precision):
    # 24^3 on [-6,6)^3, 16 x 16 x 32 rule, n = z (the closed-form case): parity with the sum
    w = synth.anisotropic_gaussian_density(24, 6.0)
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, nr=16, ntheta=16, nphi=32)
    got = _run(D, plan, w["rho"])
    ref = _oracle(_in(w["rho"], precision), w["n"], w["lo"], w["len"], w["axis"], sizes=(16, 16, 32))
    assert _report("aniso24", precision, _relinf(got, ref)) <= TOL[precision]


@pytest.mark.parametrize("precision,spread", [(0, 1), (1, 1), (1, 2)])
def test_ddi_mixture_tilted_48(D, precision, spread):
    # several tiles / columns and split (hot) tiles or shared column planes: 48^3,
    # 8-Gaussian mixture, n = (sin 30, 0, cos 30); both spreading schemes in FP32
    w = synth.gaussian_mixture_density(48, 8.0, seed=1)
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, nr=48, ntheta=24, nphi=48,
                 spread=spread)
    assert plan.info.spread == spread
    assert plan.info.spread_split_tiles > 0
    got = _run(D, plan, w["rho"])
    ref = _oracle(_in(w["rho"], precision), w["n"], w["lo"], w["len"], w["axis"], sizes=(48, 24, 48))
    assert _report(f"mix48 spread={spread}", precision, _relinf(got, ref)) <= TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_ddi_other_tile_shape_and_chunk(D, precision):
    # a different spread tiling (small chunks: many split tiles) gives the same sum
    w = synth.gaussian_mixture_density(48, 8.0, seed=4)
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, nr=48, ntheta=24, nphi=48,
                 tile=(16, 16, 16), chunk=100, spread=1)
    assert plan.info.spread_split_tiles > 4
    got = _run(D, plan, w["rho"])
    ref = _oracle(_in(w["rho"], precision), w["n"], w["lo"], w["len"], w["axis"], sizes=(48, 24, 48))
    assert _report("tiles16", precision, _relinf(got, ref)) <= TOL[precision]


@pytest.mark.parametrize("chunk", [7, 64, 100000])
def test_ddi_columns_chunk_sizes(D, chunk):
    # column spread with tiny units (most planes shared by several units and summed by the
    # reduce), default-like units, and one unit per column (its window wraps onto itself)
    w = synth.gaussian_mixture_density(48, 8.0, seed=4)
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=1, nr=48, ntheta=24, nphi=48,
                 chunk=chunk, spread=2)
    assert plan.info.spread == 2 and tuple(plan.info.tile[:2]) == (8, 8)
    got = _run(D, plan, w["rho"])
    ref = _oracle(_in(w["rho"], 1), w["n"], w["lo"], w["len"], w["axis"], sizes=(48, 24, 48))
    assert _report(f"columns chunk={chunk}", 1, _relinf(got, ref)) <= TOL[1]


@pytest.mark.parametrize("n", [(8, 8, 8), (12, 8, 16)])
def test_ddi_columns_small_fine_grids(D, n):
    # the smallest fine grids (16 cells: a footprint covers most of a column and z-windows
    # wrap), a ragged one, and the scheme the automatic choice makes for FP32 3D plans
    rng = np.random.default_rng(8)
    lo = tuple(-0.25 * v for v in n)
    ln = tuple(0.5 * v for v in n)
    X, Y, Z = synth.coords(n, lo, ln)
    rho = np.exp(-(X ** 2 + Y ** 2 + Z ** 2)) * (1 + 0.05 * rng.random(X.shape))
    plan = _plan(D, 3, n, lo, ln, (0, 0.6, 0.8), precision=1, nr=8, ntheta=6, nphi=8)
    assert plan.info.spread == 2
    got = _run(D, plan, rho)
    ref = _oracle(_in(rho, 1), n, lo, ln, (0, 0.6, 0.8), sizes=(8, 6, 8))
    assert _report(f"columns n={n}", 1, _relinf(got, ref)) <= TOL[1]


def test_ddi_columns_rejected_where_they_do_not_apply(D):
    # FP64 plans spread by tiles, and so do compensated 2D plans (2D columns have no
    # compensated variant); asking for columns there is an argument error
    with pytest.raises(D.DDIError):
        D.Plan(3, (16, 16, 16), (-1,) * 3, (2,) * 3, (0, 0, 1), precision=0, spread=2)
    with pytest.raises(D.DDIError):
        D.Plan(2, (16, 16), (-1,) * 2, (2,) * 2, (0, 0, 1), precision=1, spread=2, compensated=True)
    p = D.Plan(3, (16, 16, 16), (-1,) * 3, (2,) * 3, (0, 0, 1), precision=0)
    assert p.info.spread == 1
    p = D.Plan(2, (16, 16), (-1,) * 2, (2,) * 2, (0, 0, 1), precision=1, compensated=True)
    assert p.info.spread == 1
    p = D.Plan(2, (16, 16), (-1,) * 2, (2,) * 2, (0, 0, 1), precision=1)
    assert p.info.spread == 2 and tuple(p.info.tile[:2]) == (8, 32)


def _rho_2d(n, lo, ln, seed):
    rng = np.random.default_rng(seed)
    X, Y = synth.coords(n, lo, ln)
    return (np.exp(-((X - 0.4) ** 2 / 1.7 + (Y + 0.3) ** 2 / 0.9)) + 0.4 * np.exp(-((X + 1.5) ** 2 + (Y - 1) ** 2) / 0.6)) \
        * (1 + 0.05 * rng.random(X.shape))


@pytest.mark.parametrize("spread,chunk", [(1, 0), (2, 0), (2, 5), (2, 64), (2, 100000)])
def test_ddi_2d_spread_schemes(D, spread, chunk):
    # 2D FP32: tile spread and column spread (8-cell x columns, window along y) with the
    # default units, tiny units (most rows shared by several units and summed by the reduce),
    # and one unit per column (its window wraps onto itself)
    n, lo, ln = (64, 48), (-8.0, -6.5), (16.0, 13.0)
    axis = (np.sin(0.7), 0.0, np.cos(0.7))
    rho = _rho_2d(n, lo, ln, 5)
    plan = _plan(D, 2, n, lo, ln, axis, precision=1, spread=spread, chunk=chunk)
    assert plan.info.spread == spread
    got = _run(D, plan, rho)
    ref = _oracle(_in(rho, 1), n, lo, ln, axis, dim=2)
    assert _report(f"2d spread={spread} chunk={chunk}", 1, _relinf(got, ref)) <= TOL[1]


@pytest.mark.parametrize("n", [(8, 8), (12, 8), (8, 24)])
def test_ddi_2d_columns_small_fine_grids(D, n):
    # the smallest 2D fine grids (16 cells: a footprint covers most of a column, windows
    # wrap) and ragged ones, by the automatic choice (columns for FP32 2D plans)
    lo = tuple(-0.25 * v for v in n)
    ln = tuple(0.5 * v for v in n)
    rho = _rho_2d(n, lo, ln, 9)
    plan = _plan(D, 2, n, lo, ln, (0.6, 0.0, 0.8), precision=1)
    assert plan.info.spread == 2
    got = _run(D, plan, rho)
    ref = _oracle(_in(rho, 1), n, lo, ln, (0.6, 0.0, 0.8), dim=2)
    assert _report(f"2d columns n={n}", 1, _relinf(got, ref)) <= TOL[1]


@pytest.mark.parametrize("precision", [0, 1])
def test_ddi_ragged_anisotropic_box_two_axes(D, precision):
    # unequal sizes and spacings per axis, box not centred, two dipole axes n != m
    n, lo, ln = (32, 16, 24), (-3.0, -1.0, -5.0), (7.0, 3.0, 9.0)
    rng = np.random.default_rng(11)
    X, Y, Z = synth.coords(n, lo, ln)
    rho = np.exp(-((X - 0.3) ** 2 / 1.5 + (Y + 0.2) ** 2 / 0.7 + (Z - 0.5) ** 2 / 2.0)) * (1 + 0.1 * rng.random(X.shape))
    a = np.array([0.82778, 0.41505, -0.37751]); a /= np.linalg.norm(a)
    b = np.array([0.31180, 0.93780, -0.15214]); b /= np.linalg.norm(b)
    plan = _plan(D, 3, n, lo, ln, a, b, precision=precision, nr=20, ntheta=12, nphi=28)
    got = _run(D, plan, rho)
    ref = _oracle(_in(rho, precision), n, lo, ln, a, b, sizes=(20, 12, 28))
    assert _report("ragged two-axis", precision, _relinf(got, ref)) <= TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_ddi_smallest_grid(D, precision):
    n, lo, ln = (8, 8, 8), (-2.0, -2.0, -2.0), (4.0, 4.0, 4.0)
    rho = np.random.default_rng(3).random((8, 8, 8))
    plan = _plan(D, 3, n, lo, ln, (0, 0, 1), precision=precision)
    got = _run(D, plan, rho)
    ref = _oracle(_in(rho, precision), n, lo, ln, (0, 0, 1))
    assert _report("white noise 8^3", precision, _relinf(got, ref)) <= TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_ddi_2d_polar(D, precision):
    # the paper's printed axes (Example 2d_exmp) are rounded to 5 digits: normalise them
    setup_n = np.array([0, -0.896, 0.44404])
    setup_m = np.array([0, -0.52476, 0.85125])
    setup_n /= np.linalg.norm(setup_n)
    setup_m /= np.linalg.norm(setup_m)
    n, lo, ln = (64, 48), (-8.0, -6.0), (16.0, 12.0)
    X, Y = synth.coords(n, lo, ln)
    rho = np.exp(-(X ** 2 + Y ** 2) / 1.3) + 0.5 * np.exp(-((X - 2) ** 2 + (Y + 1) ** 2))
    plan = _plan(D, 2, n, lo, ln, setup_n, setup_m, precision=precision)
    got = _run(D, plan, rho)
    ref = _oracle(_in(rho, precision), n, lo, ln, setup_n, setup_m, dim=2)
    assert _report("2d polar 64x48", precision, _relinf(got, ref)) <= TOL[precision]


def test_ddi_zero_density_and_linearity(D):
    import torch
    n, lo, ln = (16, 16, 16), (-4.0,) * 3, (8.0,) * 3
    plan = _plan(D, 3, n, lo, ln, (0.5, 0, math.sqrt(0.75)))
    z = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    assert float(plan.apply(z).abs().max()) == 0.0
    rng = np.random.default_rng(5)
    a = torch.from_numpy(rng.random((16, 16, 16))).cuda()
    b = torch.from_numpy(rng.random((16, 16, 16))).cuda()
    pa, pb, pab = plan.apply(a), plan.apply(b), plan.apply(2 * a - 3 * b)
    assert float((pab - (2 * pa - 3 * pb)).abs().max() / pab.abs().max()) <= 1e-13


def test_ddi_in_place_and_host_path(D):
    import torch
    w = synth.gaussian_mixture_density(32, 6.0, seed=2)
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=1)
    rho = torch.from_numpy(w["rho"]).to("cuda", torch.float32)
    ref = plan.apply(rho).cpu().numpy()
    host_in = torch.from_numpy(w["rho"].astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    plan.apply_host(host_in, host_out)
    assert np.max(np.abs(host_out.numpy() - ref)) <= 1e-6 * np.max(np.abs(ref))
    plan.apply(rho, out=rho)          # rho and phi may alias
    torch.cuda.synchronize()
    assert np.max(np.abs(rho.cpu().numpy() - ref)) <= 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_density_is_reported(D, precision):
    # NaN / Inf in rho: ddi_apply with check_finite returns DDI_ERR_NONFINITE, the host
    # path reports it, an asynchronous apply leaves it for ddi_plan_check, and a finite
    # density afterwards passes (the record is cleared by each report)
    import torch
    w = synth.gaussian_mixture_density(32, 6.0, seed=3)
    rho = w["rho"].copy()
    bad = rho.copy()
    bad[5, 7, 11] = np.nan
    inf = rho.copy()
    inf[20, 1, 30] = -np.inf
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, check_finite=True)
    dt = plan.real_dtype
    for arr in (bad, inf):
        with pytest.raises(D.DDIError) as e:
            plan.apply(torch.from_numpy(arr).to("cuda", dt))
        assert e.value.status == -4
    good = plan.apply(torch.from_numpy(rho).to("cuda", dt))
    assert bool(torch.isfinite(good).all())
    # asynchronous plan: recorded, reported by the check, then cleared
    plan2 = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision)
    plan2.apply(torch.from_numpy(bad).to("cuda", dt))
    with pytest.raises(D.DDIError) as e:
        plan2.check()
    assert e.value.status == -4
    plan2.check()
    plan2.apply(torch.from_numpy(rho).to("cuda", dt))
    plan2.check()
    # host path
    host_in = torch.from_numpy(bad.astype(np.float64 if precision == 0 else np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    with pytest.raises(D.DDIError) as e:
        plan2.apply_host(host_in, host_out)
    assert e.value.status == -4
    plan2.check()


def test_compensated_fp32_plan(D):
    # compensated FP32 arithmetic (Kahan plane sums in the column spread, head + tail twiddles
    # in the fine-grid passes): parity with the oracle on the rounded input, and the same
    # result as the plain FP32 plan to the FP32 path's tolerance
    import torch
    w = synth.gaussian_mixture_density(48, 8.0, seed=1)
    kw = dict(nr=48, ntheta=24, nphi=48)
    ref = _oracle(_in(w["rho"], 1), w["n"], w["lo"], w["len"], w["axis"], sizes=(48, 24, 48))
    pc = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=1, compensated=True, **kw)
    pp = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=1, **kw)
    gc, gp = _run(D, pc, w["rho"]), _run(D, pp, w["rho"])
    ec, ep = _relinf(gc, ref), _relinf(gp, ref)
    print(f"[compensated mix48] rel err {ec:.3e}, plain {ep:.3e}")
    assert ec <= TOL[1] and _relinf(gc, gp) <= TOL[1]


def test_nonunit_axis_rejected(D):
    with pytest.raises(D.DDIError):
        D.Plan(3, (16, 16, 16), (-1,) * 3, (2,) * 3, (0, 0, 2))


def _config2():
    return synth.gaussian_mixture_density(128, 12.0, seed=0), dict(nr=128, ntheta=64, nphi=128)


@pytest.fixture(scope="module")
def full_ref():
    # oracle rhohat at all 1,048,576 nodes of the 128^3 workload (the type-2 sum, ~1 min on
    # the host); Phi at sampled grid points then costs M per point
    w, sizes = _config2()
    t = qd.plan_tables(3, w["n"], w["len"], w["axis"], **sizes)
    rh = nudft.type2(w["rho"], t["k"], w["n"], w["lo"], w["len"], block=512)
    return w, sizes, t, rh


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_ddi_sampled_points(D, full_ref, precision):
    # the timed 128^3 workload, through ddi_apply, at 1000 sampled grid points
    import torch
    w, sizes, t, rh = full_ref
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, **sizes)
    phi = plan.apply(torch.from_numpy(w["rho"]).to("cuda", plan.real_dtype)).double().cpu().numpy()
    rng = np.random.default_rng(7)
    idx = rng.integers(0, 128, size=(1000, 3))
    idx[:8] = [[64, 64, 64], [0, 0, 0], [127, 127, 127], [60, 70, 64], [64, 60, 70], [70, 64, 60], [1, 64, 127],
               [127, 0, 64]]
    pts = np.stack([w["lo"][d] + idx[:, d] * (w["len"][d] / 128) for d in range(3)], axis=1)
    ref = nudft.type1_at(t["W"] * rh, t["k"], pts)
    got = phi[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert _report("128^3 sampled points", precision, _relinf(got, ref)) <= TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_type2_sampled_nodes(D, full_ref, precision):
    # stage check: c_q = 2 h^3 W_q f_q at 3000 sampled nodes.  FP64: relative 1e-12.  FP32:
    # against the type-2 sum of the FP32-rounded density, with an absolute bound: the FP32
    # forward path (deconvolution product, FFT of (2N)^3 points in log2((2N)^3) stages, w^3 taps)
    # leaves f_q = sum_j rho_j e^{-i k_q.x_j} with an error of a few 2^-24 sum|rho| at every node,
    # and c_q scales it by 2 h^3 |W_q|, which carries the Jacobian |k|^2; where f_q has decayed
    # (|k| large) c_q is that noise alone, so no relative bound holds node by node.  Bound:
    # |c_q - ref_q| <= K 2^-24 sum|rho| 2 h^3 |W_q|, K = log2((2N)^3) + w + 2
    import torch
    w, sizes, t, rh = full_ref
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, **sizes)
    rho = torch.from_numpy(w["rho"]).to("cuda", plan.real_dtype)
    c = plan.type2(rho).cpu().numpy().astype(np.complex128)
    order = plan.node_order()
    sel = np.random.default_rng(0).choice(len(order), 3000, replace=False)
    q = order[sel]
    centre = np.array([w["lo"][d] + w["len"][d] / 2 for d in range(3)])
    rq = rh[q] if precision == 0 else nudft.type2(_in(w["rho"], 1), t["k"][q], w["n"], w["lo"], w["len"], block=512)
    ref = 2.0 * t["W"][q] * rq * np.exp(1j * (t["k"][q] @ centre))
    if precision == 0:
        err = np.max(np.abs(c[sel] - ref)) / np.max(np.abs(ref))
        assert _report("128^3 type-2 stage", precision, err) <= TOL[precision], err
    else:
        h3 = float(np.prod([w["len"][d] / 128 for d in range(3)]))
        bound = 2.0 * h3 * np.abs(t["W"][q]) * np.sum(np.abs(_in(w["rho"], 1))) * 2.0 ** -24
        K = math.log2(256.0 ** 3) + plan.info.width + 2
        ratio = float(np.max(np.abs(c[sel] - ref) / bound))
        rel = float(np.max(np.abs(c[sel] - ref)) / np.max(np.abs(ref)))
        print(f"[128^3 type-2 stage prec=1] error {ratio:.2f} x 2^-24 sum|rho| 2 h^3 |W_q| (bound K = {K:.0f}); "
              f"relative to max |c| {rel:.2e}")
        assert ratio <= K


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_type1_sampled_points(D, full_ref, precision):
    import torch
    w, sizes, t, _ = full_ref
    plan = _plan(D, 3, w["n"], w["lo"], w["len"], w["axis"], precision=precision, **sizes)
    mh = int(plan.info.nodes_used)
    rng = np.random.default_rng(1)
    c = (rng.standard_normal(mh) + 1j * rng.standard_normal(mh)) * 1e-3
    ct = torch.from_numpy(c).to("cuda", plan.cplx_dtype)
    phi = plan.type1(ct).double().cpu().numpy()
    order = plan.node_order()
    k = t["k"][order]
    centre = np.array([w["lo"][d] + w["len"][d] / 2 for d in range(3)])
    idx = rng.integers(0, 128, size=(400, 3))
    pts = np.stack([w["lo"][d] + idx[:, d] * (w["len"][d] / 128) for d in range(3)], axis=1)
    cin = c.astype(np.complex64).astype(np.complex128) if precision else c
    ref = nudft.type1_at(cin * np.exp(-1j * (k @ centre)), k, pts)
    got = phi[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert _report("128^3 type-1 stage (random node values)", precision, _relinf(got, ref)) <= TOL[precision]


def test_full_size_trace_identity(D):
    # Phi_x + Phi_y + Phi_z = 0 for any rho (symbols sum to zero), at the full size
    import torch
    w, sizes = _config2()
    tot = None
    mx = 0.0
    for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        plan = _plan(D, 3, w["n"], w["lo"], w["len"], e, precision=0, **sizes)
        phi = plan.apply(torch.from_numpy(w["rho"]).cuda())
        mx = max(mx, float(phi.abs().max()))
        tot = phi if tot is None else tot + phi
        del plan
    assert float(tot.abs().max()) <= 1e-12 * mx

"""GPU batches of DDI evaluations (ddi_batch_*) and the spread-tile autotuner, through
the C ABI, against the FP64 oracle and against single-plan ddi_apply.

Tolerances as for single plans (relative L-infinity, normalised by max |oracle|):
1e-12 for FP64 items, 1e-6 for FP32 items."""
import math

import numpy as np
import pytest

from oracle import nudft
from oracle import quadrature as qd
from paper_1504_02897_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}


def fp32_reference(it, ref):
    """The oracle on the density rounded to FP32 (what the FP32 path receives) and the
    input-rounding floor |Phi(rho32) - Phi(rho)| / max|Phi(rho)|.  FP32 items are compared
    with the rounded-input oracle.  In 3D the symbol is bounded (|Uhat| <= 2) and the FP32
    path stays below 1e-6 of it.  In 2D the weights grow like |k| up to R = pi/h: white
    rounding noise of relative size 2^-24 anywhere before the weights (the input itself,
    which the floor measures, but also the FP32 deconvolution product and the forward FFT's
    roundoff, which have the same white spectrum) is amplified by ~R, so the FP32 path's own
    error after removing the input rounding is a multiple of the floor (measured 2.2-2.7 x;
    the floor grows with N: 4.6e-7 at 128^2, 1.2e-6 at 256^2, 2.3e-6 at 512^2): 2D items are
    held to max(1e-6, 4 x floor)."""
    t = qd.plan_tables(len(it["n"]), it["n"], it["len"], it["axis"])
    r32 = nudft.ddi(it["rho"].astype(np.float32).astype(np.float64), t, it["n"], it["lo"], it["len"])
    return r32, _relinf(r32, ref)


def fp32_tol(it, floor):
    return TOL[1] if len(it["n"]) == 3 else max(TOL[1], 4.0 * floor)


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


def _desc(D, it, precision, tile=None):
    dim = len(it["n"])
    return D.make_desc(dim, it["n"], it["lo"], it["len"], it["axis"], precision=precision, tile=tile)


def _oracle(it):
    dim = len(it["n"])
    t = qd.plan_tables(dim, it["n"], it["len"], it["axis"])
    return nudft.ddi(it["rho"], t, it["n"], it["lo"], it["len"])


def _tensors(items, descs):
    import torch
    out = []
    for it, d in zip(items, descs):
        dt = torch.float64 if d.precision == 0 else torch.float32
        out.append(torch.from_numpy(np.ascontiguousarray(it["rho"])).to("cuda", dt))
    return out


def _mixed_items():
    # 2D densities shaped like the batched workload (random box, tilt, 4 Gaussians) at
    # small sizes, plus two 3D mixtures
    items = synth.batch_2d(count=6, seed=3, sizes=(32, 48, 64, 96))
    for seed, (N, L) in enumerate([(24, 6.0), (32, 8.0)]):
        it = synth.gaussian_mixture_density(N, L, seed=seed, centre=L / 3)
        a = math.radians(20.0 + 25.0 * seed)
        items.append(dict(it, axis=(math.sin(a), 0.0, math.cos(a))))
    return items


@pytest.mark.parametrize("graph", [False, True])
def test_batch_mixed_matches_oracle(D, graph):
    # mixed dims, sizes, axes and precisions in one batch, autotuned tiles
    import torch
    items = _mixed_items()
    descs = [_desc(D, it, precision=i % 2) for i, it in enumerate(items)]
    b = D.Batch(descs, graph=graph, autotune=True)
    rhos = _tensors(items, descs)
    outs = b.apply(rhos)
    torch.cuda.synchronize()
    for i, (it, d, o) in enumerate(zip(items, descs, outs)):
        assert b.infos[i].spread_tuned_ms > 0.0
        ref = _oracle(it)
        tol = TOL[d.precision]
        if d.precision == 1:
            ref, floor = fp32_reference(it, ref)
            tol = fp32_tol(it, floor)
        err = _relinf(o.double().cpu().numpy(), ref)
        print(f"[batch item {i} n={it['n']} prec={d.precision}] rel err {err:.3e} (tol {tol:.1e})")
        assert err <= tol, (i, it["n"], d.precision, err)
    b.close()


def test_batch_bitwise_equals_single_plans(D):
    # same tiles (built-in choice, no autotuning): the batch runs the same kernels with
    # the same work lists as ddi_apply, so every item is bit-identical
    import torch
    items = _mixed_items()
    descs = [_desc(D, it, precision=(i + 1) % 2) for i, it in enumerate(items)]
    b = D.Batch(descs, graph=True, autotune=False)
    rhos = _tensors(items, descs)
    outs = b.apply(rhos)
    torch.cuda.synchronize()
    for i, (it, d) in enumerate(zip(items, descs)):
        dim = len(it["n"])
        p = D.Plan(dim, it["n"], it["lo"], it["len"], it["axis"], precision=d.precision)
        assert tuple(p.info.tile) == tuple(b.infos[i].tile)
        ref = p.apply(rhos[i])
        torch.cuda.synchronize()
        assert torch.equal(ref, outs[i]), i
        p.close()
    b.close()


def test_batch_graph_replay_and_new_pointers(D):
    import torch
    items = synth.batch_2d(count=5, seed=7, sizes=(32, 64, 128))
    descs = [_desc(D, it, precision=1) for it in items]
    b = D.Batch(descs, graph=True, autotune=True)
    rhos = _tensors(items, descs)
    outs = [torch.empty_like(r) for r in rhos]
    b.apply(rhos, outs)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    b.apply(rhos, outs)  # same pointers: replay
    torch.cuda.synchronize()
    assert b.graph_stats() == (1, 2)
    for f, o in zip(first, outs):
        assert torch.equal(f, o)
    # new output buffers and an in-place item: the graph is recorded again
    outs2 = [torch.empty_like(r) for r in rhos]
    rin = rhos[2].clone()
    outs2[2] = rin
    rhos2 = list(rhos)
    rhos2[2] = rin
    b.apply(rhos2, outs2)
    torch.cuda.synchronize()
    assert b.graph_stats() == (2, 3)
    for f, o in zip(first, outs2):
        assert torch.equal(f, o)
    # replays keep following the inputs' contents
    rhos[0].mul_(2.0)
    b.apply(rhos2, outs2)
    torch.cuda.synchronize()
    assert b.graph_stats() == (2, 4)
    assert _relinf(outs2[0].double().cpu().numpy(), 2.0 * first[0].double().cpu().numpy()) <= 1e-6
    b.close()


def test_batch_rejects_bad_input(D):
    import torch
    items = synth.batch_2d(count=2, seed=1, sizes=(32,))
    descs = [_desc(D, it, precision=1) for it in items]
    bad = D.make_desc(2, (30, 32), (-4.0, -4.0), (8.0, 8.0), (1.0, 0.0, 0.0), precision=1)
    with pytest.raises(D.DDIError) as e:
        D.Batch(descs + [bad])
    assert "item 2" in str(e.value)
    b = D.Batch(descs, graph=False, autotune=False)
    rhos = _tensors(items, descs)
    with pytest.raises(ValueError):
        b.apply(rhos[:1])
    with pytest.raises(ValueError):
        b.apply([rhos[0], rhos[1].double()])
    b.close()


def test_autotuned_plan_and_cache(D):
    # tile[0] < 0: the plan's spread tile is picked by timing candidates; a second plan of
    # the same node-set shape (other box length and axis) reuses the cached choice
    import torch
    N, L = 48, 9.0
    it = synth.gaussian_mixture_density(N, L, seed=4, centre=3.0)
    n, lo, ln, rho = it["n"], it["lo"], it["len"], it["rho"]
    p1 = D.Plan(3, n, lo, ln, (0.0, 0.6, 0.8), precision=1, tile=(-1, 0, 0))
    assert p1.info.spread_tuned_ms > 0.0
    got = p1.apply(torch.from_numpy(rho).to("cuda", torch.float32))
    torch.cuda.synchronize()
    t = qd.plan_tables(3, n, ln, (0.0, 0.6, 0.8))
    ref = nudft.ddi(rho.astype(np.float32).astype(np.float64), t, n, lo, ln)
    assert _relinf(got.double().cpu().numpy(), ref) <= TOL[1]
    n2, lo2, ln2 = synth.box(N, 11.0, 3)
    p2 = D.Plan(3, n2, lo2, ln2, (1.0, 0.0, 0.0), precision=1, tile=(-1, 0, 0))
    assert tuple(p2.info.tile) == tuple(p1.info.tile)
    assert p2.info.spread_tuned_ms == p1.info.spread_tuned_ms
    p1.close()
    p2.close()


def test_batch_1024_item_stages(D):
    # a 1024^2 item of the batched workload through its single plan (batch items compute the
    # same bits as their single plans): the type-2 stage at 256 sampled nodes and the type-1
    # stage (seeded random node values) at 256 sampled grid points, each against the oracle's
    # per-node / per-point sums on the FP32-rounded inputs.
    # The type-2 stage carries an absolute error, not a relative one: the FP32 forward path
    # (deconvolution product, 2D FFT of (2N)^2 points in log2((2N)^2) stages, w x w taps) leaves
    # the sum f_q = sum_j rho_j e^{-i k_q.x_j} with an error of a few 2^-24 sum|rho|, the same at
    # every node, and c_q = 2 h^2 W_q f_q scales it by 2 h^2 |W_q|, which grows like |k| to
    # R = pi/h; where f_q itself has decayed (|k| large) c_q is that noise alone.  Bound:
    # |c_q - ref_q| <= K 2^-24 sum|rho| 2 h^2 |W_q| with K = log2((2N)^2) + w + 2 (a rounding's
    # worth per FFT stage and per tap row)
    import torch
    it = next(x for x in synth.batch_2d(count=96, seed=0) if x["n"][0] == 1024)
    plan = D.Plan(2, it["n"], it["lo"], it["len"], it["axis"], precision=1)
    t = qd.plan_tables(2, it["n"], it["len"], it["axis"])
    order = plan.node_order()
    centre = np.array([it["lo"][d] + it["len"][d] / 2 for d in range(2)])
    rng = np.random.default_rng(13)
    # type 2: c_q = 2 h^2 W_q f_q
    c = plan.type2(torch.from_numpy(it["rho"]).to("cuda", torch.float32)).cpu().numpy().astype(np.complex128)
    sel = rng.choice(len(order), 256, replace=False)
    q = order[sel]
    r32 = it["rho"].astype(np.float32).astype(np.float64)
    ref = 2.0 * t["W"][q] * nudft.type2(r32, t["k"][q], it["n"], it["lo"], it["len"]) * np.exp(1j * (t["k"][q] @ centre))
    h2 = (it["len"][0] / 1024) * (it["len"][1] / 1024)
    scale = 2.0 * h2 * np.abs(t["W"][q]) * np.sum(np.abs(r32))
    K = math.log2(2048.0 * 2048.0) + plan.info.width + 2
    e2 = float(np.max(np.abs(c[sel] - ref) / scale) / 2.0 ** -24)   # in units of 2^-24
    # type 1 of random node values (rounded to complex64, the plan's precision)
    mh = int(plan.info.nodes_used)
    cv = ((rng.standard_normal(mh) + 1j * rng.standard_normal(mh)) * 1e-3).astype(np.complex64)
    phi = plan.type1(torch.from_numpy(cv).cuda()).double().cpu().numpy()
    k = t["k"][order]
    idx = rng.integers(0, 1024, size=(256, 2))
    pts = np.stack([it["lo"][d] + idx[:, d] * (it["len"][d] / 1024) for d in range(2)], axis=1)
    ref1 = nudft.type1_at(cv.astype(np.complex128) * np.exp(-1j * (k @ centre)), k, pts)
    e1 = _relinf(phi[idx[:, 1], idx[:, 0]], ref1)
    print(f"[batch 1024^2 item] type-2 stage error {e2:.2f} x 2^-24 sum|rho| 2 h^2 |W_q| (bound K = {K:.0f}); "
          f"type-1 stage rel err {e1:.3e}")
    assert e1 <= TOL[1]
    assert e2 <= K
    plan.close()


def test_batch_2d_1024_trace_identity(D):
    # 2D trace identity at the largest batched size: with m = n, the symbol summed over
    # n = e_x, e_y, e_z is 3/2 [(k_x^2 + k_y^2)/|k| - |k|] = 0 at every node, so the three
    # potentials of one density sum to zero up to the NUFFT error
    import torch
    it = synth.batch_2d(count=1, seed=11, sizes=(1024,))[0]
    items = [dict(it, axis=a) for a in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))]
    descs = [_desc(D, x, precision=1) for x in items]
    b = D.Batch(descs, graph=True, autotune=True)
    outs = b.apply(_tensors(items, descs))
    torch.cuda.synchronize()
    s = (outs[0].double() + outs[1].double() + outs[2].double()).abs().max().item()
    scale = max(o.double().abs().max().item() for o in outs)
    assert s / scale <= 2e-6
    b.close()


def test_batch_96_densities_2d(D):
    # the batched 2D workload: 96 densities, N in {128, 256, 512, 1024}, box length
    # U[8, 16], tilt U[0, 90] degrees, 4 Gaussians each, quadrature 2N x 2N, FP32,
    # autotuned tiles, one recorded graph.  Oracle parity on a subset: four 128^2 items and one
    # 256^2 item on the whole grid, two 512^2 items and one 1024^2 item at 200 sampled grid
    # points, against the oracle on the FP32-rounded density (fp32_reference, fp32_tol).
    import torch
    items = synth.batch_2d(count=96, seed=0)
    descs = [_desc(D, it, precision=1) for it in items]
    b = D.Batch(descs, graph=True, autotune=True)
    rhos = _tensors(items, descs)
    outs = b.apply(rhos)
    torch.cuda.synchronize()
    assert b.graph_stats() == (1, 1)
    for o in outs:
        assert bool(torch.isfinite(o).all())
    small = [i for i, it in enumerate(items) if it["n"][0] == 128][:4]
    small += [i for i, it in enumerate(items) if it["n"][0] == 256][:1]
    for i in small:
        ref, floor = fp32_reference(items[i], _oracle(items[i]))
        err = _relinf(outs[i].double().cpu().numpy(), ref)
        tol = fp32_tol(items[i], floor)
        print(f"[batch96 item {i} n={items[i]['n']}] rel err {err:.3e} vs rounded input (floor {floor:.2e}, "
              f"tol {tol:.1e})")
        assert err <= tol, (i, items[i]["n"], err, floor)
    # two 512^2 items at 200 sampled grid points: the oracle's type-2 sum at all 4 N^2 nodes
    # (for the density and for its FP32 rounding), then the type-1 sum at the points
    large = [i for i, it in enumerate(items) if it["n"][0] == 512][:2]
    rng = np.random.default_rng(12)
    for i in large:
        it = items[i]
        t = qd.plan_tables(2, it["n"], it["len"], it["axis"])
        N = it["n"][0]
        idx = rng.integers(0, N, size=(200, 2))
        pts = np.stack([it["lo"][d] + idx[:, d] * (it["len"][d] / N) for d in range(2)], axis=1)
        refs = []
        for rho in (it["rho"], it["rho"].astype(np.float32).astype(np.float64)):
            rh = nudft.type2(rho, t["k"], it["n"], it["lo"], it["len"], block=1024)
            refs.append(nudft.type1_at(t["W"] * rh, t["k"], pts))
        floor = _relinf(refs[1], refs[0])
        got = outs[i].double().cpu().numpy()[idx[:, 1], idx[:, 0]]
        err = _relinf(got, refs[1])
        tol = fp32_tol(it, floor)
        print(f"[batch96 item {i} n={it['n']}] rel err {err:.3e} at 200 points vs rounded input "
              f"(floor {floor:.2e}, tol {tol:.1e})")
        assert err <= tol, (i, it["n"], err, floor)
    b.close()

"""GPU parity of the ellipsoidal rule on heterogeneous boxes (the thin domains D_eps of
Sec. 2.1, h_z = eps h_x in 3D and h_y = eps h_x in 2D; ``ellipsoid=True``) against the FP64
oracle with the same rule.  Tolerances: 1e-12 (FP64 plans); FP32 plans 1e-6, or 8x the
change of the exact sum when the density is rounded to FP32 where that is larger (in 2D the
symbol grows like |k| up to pi / h_y)."""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import nudft
from oracle import quadrature as qd

pytestmark = pytest.mark.gpu

N_2D = np.array([0, -0.896, 0.44404]) / np.linalg.norm([0, -0.896, 0.44404])   # Example 2d_exmp
M_2D = np.array([0, -0.52476, 0.85125]) / np.linalg.norm([0, -0.52476, 0.85125])


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


def _thin(dim, L, eps, hx):
    n = (int(round(2 * L / hx)),) * dim
    lo = (-L,) * (dim - 1) + (-eps * L,)
    ln = (2 * L,) * (dim - 1) + (2 * eps * L,)
    ax = [lo[d] + np.arange(n[d]) * (ln[d] / n[d]) for d in range(dim)]
    mesh = list(reversed(np.meshgrid(*reversed(ax), indexing="ij")))
    pts = np.stack([g.ravel() for g in mesh], axis=1)
    s2 = [2.0] * (dim - 1) + [2.0 * eps * eps]
    rho = cf.gaussian_density(pts, s2, [0.0] * dim, 1.0).reshape(mesh[0].shape)
    return n, lo, ln, rho


CASES = {
    # Table ani_3d_cs1's density on [-8,8]^2 x [-2,2], tilted axis
    "3d": dict(dim=3, geo=(8.0, 0.25, 0.5), axis=(math.sin(0.3), 0.0, math.cos(0.3)), m=None,
               sizes=dict(nr=48, ntheta=32, nphi=48)),
    # Table ani_2d's density on [-8,8] x [-2,2], the axes of Example 2d_exmp
    "2d": dict(dim=2, geo=(8.0, 0.25, 0.25), axis=N_2D, m=M_2D, sizes=dict(nr=96, nphi=384)),
}


@pytest.mark.parametrize("name", ["3d", "2d"])
@pytest.mark.parametrize("precision", [0, 1])
def test_thin_box_matches_oracle(D, name, precision):
    import torch
    c = CASES[name]
    dim = c["dim"]
    n, lo, ln, rho = _thin(dim, *c["geo"])
    plan = D.Plan(dim, n, lo, ln, c["axis"], c["m"], precision=precision, ellipsoid=True, **c["sizes"])
    got = plan.apply(torch.from_numpy(rho).to("cuda", plan.real_dtype)).double().cpu().numpy()
    t = qd.plan_tables(dim, n, ln, c["axis"], c["m"], ellipsoid=True, **c["sizes"])
    ref = nudft.ddi(rho, t, n, lo, ln)
    tol = 1e-12
    if precision:
        # FP32: against the oracle on the FP32-rounded density (what the path receives); in
        # 2D the symbol grows like |k| (here up to pi/h_y = 50), so white rounding noise before
        # the weights (the FP32 deconvolution product, the forward FFT) is amplified like the
        # input rounding: max(1e-6, 4 x the input-rounding floor), see tests/test_gpu_batch.py
        r32 = nudft.ddi(rho.astype(np.float32).astype(np.float64), t, n, lo, ln)
        floor = _relinf(r32, ref)
        ref = r32
        tol = 1e-6 if dim == 3 else max(1e-6, 4.0 * floor)
    err = _relinf(got, ref)
    print(f"[thin {name} prec={precision}] rel err {err:.3e} (tol {tol:.1e})")
    assert err <= tol


def test_thin_box_set_axes_equals_fresh_plan(D):
    # the stored symbol direction of an ellipsoidal node is that of k, so rebuilt weights
    # are those of a fresh plan bit for bit
    import torch
    c = CASES["3d"]
    n, lo, ln, rho = _thin(3, *c["geo"])
    plan = D.Plan(3, n, lo, ln, (0.0, 0.0, 1.0), precision=1, ellipsoid=True, **c["sizes"])
    r = torch.from_numpy(rho).to("cuda", torch.float32)
    plan.apply(r)
    a1 = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    plan.set_axes(tuple(a1))
    got = plan.apply(r)
    fresh = D.Plan(3, n, lo, ln, tuple(a1), precision=1, ellipsoid=True, **c["sizes"])
    ref = fresh.apply(r)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)

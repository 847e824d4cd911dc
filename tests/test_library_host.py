"""Host-side checks of the CUDA library (no GPU needed): it builds, loads, exports every
function include/ddi.h declares, and its host plan builder reproduces the oracle's
quadrature tables bit for bit (same rule, same evaluation order, -ffp-contract=off)."""
import math
import os
import re

import numpy as np
import pytest

from oracle import quadrature as qd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1504_02897_gb300 import build, ddi
    build.build()
    return ddi


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)
    return names


def test_exports_every_declared_symbol(lib):
    import ctypes
    handle = ctypes.CDLL(lib.lib_path())
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(handle, name), name
    assert set(lib.EXPORTS) <= set(declared)


def test_status_strings(lib):
    L = lib.load()
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.ddi_status_str(s) and b"unknown" not in L.ddi_status_str(s)


CASES = [
    dict(dim=3, n=(24, 24, 24), lo=(-6, -6, -6), length=(12, 12, 12), axis=(0, 0, 1), sizes=(16, 16, 32)),
    dict(dim=3, n=(32, 16, 64), lo=(-4, -2, -8), length=(8, 3, 16), axis=(0.5, 0, math.sqrt(0.75)), sizes=(0, 0, 0)),
    dict(dim=3, n=(128, 128, 128), lo=(-12,) * 3, length=(24,) * 3,
         axis=(math.sin(math.radians(30)), 0, math.cos(math.radians(30))), sizes=(128, 64, 128)),
    dict(dim=2, n=(256, 256), lo=(-10, -10), length=(20, 20), axis=(0.3, 0.0, math.sqrt(0.91)), sizes=(0, 0, 0)),
    dict(dim=2, n=(64, 32), lo=(-8, -4), length=(16, 8), axis=(0, -0.896, 0.44404), m=(0, -0.52476, 0.85125),
         sizes=(40, 0, 50)),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_tables_bitwise_equal_oracle(lib, case, precision):
    axis = np.array(case["axis"], float)
    axis = axis / np.linalg.norm(axis)
    m = case.get("m")
    if m is not None:
        m = np.array(m, float)
        m = m / np.linalg.norm(m)
    nr, nt, npp = case["sizes"]
    desc = lib.make_desc(case["dim"], case["n"], case["lo"], case["length"], axis, m, nr=nr, ntheta=nt, nphi=npp,
                         precision=precision)
    k, W, l0 = lib.quadrature_tables(desc)
    ref = qd.plan_tables(case["dim"], case["n"], case["length"], axis, m, nr=nr, ntheta=nt, nphi=npp)
    assert k.shape == ref["k"].shape
    assert np.array_equal(k, ref["k"]), np.max(np.abs(k - ref["k"]))
    assert np.array_equal(W, ref["W"]), np.max(np.abs(W - ref["W"]))
    width = {0: 14, 1: 8}[precision]
    nf = [2 * v for v in case["n"]]
    ref_l0 = qd.fine_grid_start(ref["k"], ref["h"], nf, width)
    assert np.array_equal(l0.astype(np.int64), ref_l0)


def test_gauss_legendre_bitwise_large(lib):
    # 2D default radial rule at N = 1024 uses 2048 Gauss-Legendre nodes
    desc = lib.make_desc(2, (1024, 1024), (-8, -8), (16, 16), (1, 0, 0), nr=2048, nphi=2)
    k, W, _ = lib.quadrature_tables(desc)
    ref = qd.plan_tables(2, (1024, 1024), (16, 16), (1, 0, 0), nr=2048, nphi=2)
    assert np.array_equal(k, ref["k"]) and np.array_equal(W, ref["W"])


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(n=(20, 16, 16)), dict(n=(4, 16, 16)), dict(axis=(1, 1, 0)), dict(nphi=7),
    dict(length=(0, 1, 1)), dict(precision=3),
])
def test_descriptor_validation(lib, bad):
    args = dict(dim=3, n=(16, 16, 16), lo=(-1, -1, -1), length=(2, 2, 2), axis=(0, 0, 1), nphi=0, precision=0)
    args.update(bad)
    desc = lib.make_desc(args["dim"], args["n"], args["lo"], args["length"], args["axis"], nphi=args["nphi"],
                         precision=args["precision"])
    with pytest.raises(lib.DDIError) as e:
        lib.quadrature_tables(desc)
    assert e.value.status == -1
    assert len(str(e.value)) > 20


def test_null_arguments_are_rejected_before_any_device_work(lib):
    # argument checks of the entry points that take handles come before any CUDA call,
    # so they answer DDI_ERR_ARG (or a documented no-op) on a machine without a GPU
    import ctypes
    L = lib.load()
    n = (ctypes.c_double * 3)(0.0, 0.0, 1.0)
    assert L.ddi_plan_set_axes(None, n, None, None) == -1
    assert L.ddi_plan_set_axes(ctypes.c_void_p(1), None, None, None) == -1
    assert L.ddi_batch_size(None) == 0
    assert L.ddi_batch_destroy(None) == 0
    assert L.ddi_batch_apply(None, None, None, None) == -1
    assert L.ddi_batch_get_info(None, 0, None) == -1
    assert L.ddi_batch_graph_stats(None, None, None) == -1
    assert L.ddi_plan_check(None, None) == -1
    out = ctypes.c_void_p()
    desc = lib.make_desc(3, (16, 16, 16), (-1, -1, -1), (2, 2, 2), (0, 0, 1))
    assert L.ddi_batch_create(None, ctypes.byref(desc), 1, 0, None) == -1
    assert L.ddi_batch_create(ctypes.byref(out), ctypes.byref(desc), 0, 0, None) == -1
    assert L.ddi_batch_create(ctypes.byref(out), ctypes.byref(desc), 1, 8, None) == -1  # unknown flag
    assert b"flags" in L.ddi_last_error()


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as C99 and links against the library
    import shutil
    import subprocess
    from paper_1504_02897_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "ddi.h"\n#include <string.h>\n'
                   'int main(void) { ddi_plan_desc d; memset(&d, 0, sizeof d);\n'
                   '  return strlen(ddi_status_str(DDI_ERR_ARG)) > 0 && ddi_batch_size(0) == 0 ? 0 : 1; }\n')
    exe = tmp_path / "use"
    lib = build.LIB
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), lib,
                        "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0


def test_binding_structs_match_the_c_layout(tmp_path):
    # the ctypes mirrors of the header's structs have the C sizes and field offsets
    import ctypes
    import shutil
    import subprocess
    from paper_1504_02897_gb300 import ddi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = [("ddi_plan_desc", ddi.PlanDesc), ("ddi_plan_info", ddi.PlanInfo), ("gpe_stats", ddi.GpeStats),
              ("gpe_nonlinearity", ddi.GpeNonlinearity)]
    lines = ['#include "ddi.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for cname, _ in checks:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
    for cname, py in checks:
        for f, _ in py._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(py) for _, py in checks]
    for _, py in checks:
        want += [getattr(py, f).offset for f, _ in py._fields_]
    assert got == want


# ---- the split algorithm's ball tables (Sec. 2.1, Eq. 3.9) ---------------------------------------

SPLIT_CASES = [
    dict(n=(32, 32, 32), lo=(-8,) * 3, length=(16,) * 3, axis=(0, 0, 1), m=None, k0=0.8, sizes=(48, 32, 64)),
    dict(n=(64, 32, 48), lo=(-6, -3, -5), length=(12, 7, 10), axis=(0.5, 0, math.sqrt(0.75)),
         m=(0.6, 0.0, 0.8), k0=1.3, sizes=(24, 16, 40)),
]


@pytest.mark.parametrize("case", SPLIT_CASES)
def test_split_ball_tables_match_oracle(lib, case):
    # nodes bit for bit (the spherical rule on |k| <= 6 k0); weights W_q q(k_q) to a few ulp
    # (the library folds the window into the weight before the symbol, the oracle after it)
    from oracle import split
    axis = np.array(case["axis"], float)
    axis /= np.linalg.norm(axis)
    m = None if case["m"] is None else np.array(case["m"], float) / np.linalg.norm(case["m"])
    nr, nt, npp = case["sizes"]
    desc = lib.make_desc(3, case["n"], case["lo"], case["length"], axis, m, nr=nr, ntheta=nt, nphi=npp,
                         precision=0, split_k0=case["k0"])
    k, W, l0 = lib.quadrature_tables(desc)
    ref = split.ball_tables(case["n"], case["length"], axis, m, k0=case["k0"], nr=nr, ntheta=nt, nphi=npp)
    assert np.array_equal(k, ref["k"])
    assert np.max(np.abs(W - ref["W"])) <= 1e-15 * np.max(np.abs(ref["W"]))
    assert np.all(np.abs(W - ref["W"]) <= 4 * np.spacing(np.abs(ref["W"])))
    h = [case["length"][d] / case["n"][d] for d in range(3)]
    assert np.array_equal(l0.astype(np.int64), qd.fine_grid_start(ref["k"], h, [2 * v for v in case["n"]], 14))


def test_split_defaults(lib):
    # k0 = 9.6 / min len, ball 6 k0, sizes 0.48 K / 0.32 K / 0.64 K rounded up to multiples of 8,
    # K = 6 k0 times the box diagonal: on [-12, 12)^3, k0 = 0.4, K = 2.4 * 24 sqrt(3) = 99.8
    desc = lib.make_desc(3, (128,) * 3, (-12,) * 3, (24,) * 3, (0.5, 0, math.sqrt(0.75)), precision=1, split_k0=-1)
    k, W, _ = lib.quadrature_tables(desc)
    assert k.shape == (48 * 32 * 64, 3)
    r = np.linalg.norm(k, axis=1)
    assert r.max() < 2.4 and r.max() > 2.39
    ref = lib.make_desc(3, (128,) * 3, (-12,) * 3, (24,) * 3, (0.5, 0, math.sqrt(0.75)), precision=1,
                        split_k0=9.6 / 24, kmax=6 * (9.6 / 24), nr=48, ntheta=32, nphi=64)
    k2, W2, _ = lib.quadrature_tables(ref)
    assert np.array_equal(k, k2) and np.array_equal(W, W2)


@pytest.mark.parametrize("bad", [
    dict(dim=2, n=(64, 64), split_k0=1.0),            # 3D only
    dict(n=(8, 8, 8), split_k0=-1.0),                 # 6 k0 beyond the band of a coarse grid
    dict(split_k0=float("nan")),
    dict(split_k0=1.0, kmax=100.0),
])
def test_split_descriptor_validation(lib, bad):
    args = dict(dim=3, n=(32, 32, 32), lo=(-8,) * 3, length=(16,) * 3, split_k0=0.0, kmax=0.0)
    args.update(bad)
    dim = args["dim"]
    desc = lib.make_desc(dim, args["n"], args["lo"][:dim], args["length"][:dim], (0, 0, 1), precision=0,
                         split_k0=args["split_k0"], kmax=args["kmax"])
    with pytest.raises(lib.DDIError) as e:
        lib.quadrature_tables(desc)
    assert e.value.status == -1


# ---- the ellipsoidal rule for heterogeneous boxes ------------------------------------------------

ELL_CASES = [
    # thin 3D box D_eps = [-8,8]^2 x [-2,2] (eps = 1/4, h_z = h_x / 4), default sizes (32, 64, 32)
    dict(dim=3, n=(32, 32, 32), lo=(-8, -8, -2), length=(16, 16, 4), axis=(0, 0, 1), m=None, sizes=(0, 0, 0)),
    # ragged 3D box, two axes, explicit sizes
    dict(dim=3, n=(32, 16, 64), lo=(-4, -2, -8), length=(8, 3, 16), axis=(0.5, 0, math.sqrt(0.75)),
         m=(0.6, 0.0, 0.8), sizes=(24, 20, 36)),
    # thin 2D rectangle [-8,8] x [-2,2] with the axes of Example 2d_exmp, default sizes (128, -, 512)
    dict(dim=2, n=(64, 64), lo=(-8, -2), length=(16, 4), axis=(0, -0.896, 0.44404), m=(0, -0.52476, 0.85125),
         sizes=(0, 0, 0)),
]


@pytest.mark.parametrize("case", ELL_CASES)
def test_ellipsoid_tables_bitwise_equal_oracle(lib, case):
    axis = np.array(case["axis"], float)
    axis /= np.linalg.norm(axis)
    m = None if case["m"] is None else np.array(case["m"], float) / np.linalg.norm(case["m"])
    nr, nt, npp = case["sizes"]
    desc = lib.make_desc(case["dim"], case["n"], case["lo"], case["length"], axis, m, nr=nr, ntheta=nt, nphi=npp,
                         precision=0, ellipsoid=True)
    k, W, l0 = lib.quadrature_tables(desc)
    ref = qd.plan_tables(case["dim"], case["n"], case["length"], axis, m, nr=nr, ntheta=nt, nphi=npp, ellipsoid=True)
    assert k.shape == ref["k"].shape
    assert np.array_equal(k, ref["k"]), np.max(np.abs(k - ref["k"]))
    assert np.array_equal(W, ref["W"]), np.max(np.abs(W - ref["W"]))
    nf = [2 * v for v in case["n"]]
    assert np.array_equal(l0.astype(np.int64), qd.fine_grid_start(ref["k"], ref["h"], nf, 14))
    # every node stays inside its own axis' band |k_d| <= pi / h_d
    for d in range(case["dim"]):
        assert np.max(np.abs(k[:, d])) * ref["h"][d] <= math.pi * (1 + 1e-15)


def test_ellipsoid_defaults(lib):
    desc = lib.make_desc(3, (32, 32, 32), (-8, -8, -2), (16, 16, 4), (0, 0, 1), ellipsoid=True)
    k, _, _ = lib.quadrature_tables(desc)
    assert k.shape[0] == 32 * 64 * 32          # ceil(32/2 * 4) polar nodes
    desc = lib.make_desc(2, (64, 64), (-8, -2), (16, 4), (1, 0, 0), ellipsoid=True)
    k, _, _ = lib.quadrature_tables(desc)
    assert k.shape[0] == 128 * 512             # 2 ceil(64 * 4) azimuthal nodes


@pytest.mark.parametrize("bad", [dict(ellipsoid=2), dict(ellipsoid=1, split_k0=1.0)])
def test_ellipsoid_descriptor_validation(lib, bad):
    desc = lib.make_desc(3, (32, 32, 32), (-8,) * 3, (16,) * 3, (0, 0, 1), split_k0=bad.get("split_k0", 0.0))
    desc.ellipsoid = bad["ellipsoid"]
    with pytest.raises(lib.DDIError) as e:
        lib.quadrature_tables(desc)
    assert e.value.status == -1


# ---- ddi_plan_describe: the plan's derived parameters without a GPU ---------------------------------

def test_describe_matches_the_tables_and_defaults(lib):
    desc = lib.make_desc(3, (128,) * 3, (-12,) * 3, (24,) * 3, (0.5, 0, math.sqrt(0.75)), precision=1)
    info = lib.describe(desc)
    assert (info.nr, info.ntheta, info.nphi) == (128, 64, 128) and info.nodes == 128 * 64 * 128
    assert info.nodes_used == info.nodes // 2 and list(info.nf) == [256] * 3
    assert info.width == 8 and info.kmax == pytest.approx(math.pi / 0.1875)
    assert info.split_k0 == 0.0 and list(info.band) == [0, 0] and info.ellipsoid == 0
    info64 = lib.describe(lib.make_desc(2, (64, 32), (-8, -4), (16, 8), (1, 0, 0), precision=0, ellipsoid=True))
    assert info64.width == 14 and info64.ellipsoid == 1 and list(info64.nf) == [128, 64, 1]
    import ctypes
    assert lib.load().ddi_plan_describe(ctypes.byref(desc), None) == -1


@pytest.mark.parametrize("precision", [0, 1])
def test_split_band_holds_every_ball_tap(lib, precision):
    # the band of fine lines the ball's y/z passes transform contains every tap of every node
    # (first taps from the library's own tables), and is narrower than the axis
    desc = lib.make_desc(3, (128,) * 3, (-12,) * 3, (24,) * 3, (0.5, 0, math.sqrt(0.75)), precision=precision,
                         split_k0=-1.0)
    info = lib.describe(desc)
    assert list(info.band) == ([27, 27] if precision == 0 else [24, 24])
    _, _, l0 = lib.quadrature_tables(desc)
    w = info.width
    for a in range(2):
        assert l0[:, a].min() >= -info.band[a] and (l0[:, a] + w - 1).max() <= info.band[a]
        assert 2 * info.band[a] + 1 < info.nf[a]
    full = lib.make_desc(3, (128,) * 3, (-12,) * 3, (24,) * 3, (0.5, 0, math.sqrt(0.75)), precision=precision,
                         split_k0=-1.0, split_full_passes=True)
    assert list(lib.describe(full).band) == [0, 0]
    # a band that would cover the axis is not used
    coarse = lib.make_desc(3, (32,) * 3, (-8,) * 3, (16,) * 3, (0, 0, 1), precision=0, split_k0=0.8)
    assert list(lib.describe(coarse).band) == [0, 0]


def test_noalloc_binding_rejects_mismatched_dtypes(lib):
    # the binding checks dtypes before anything reaches the library (a complex128 psi with a
    # float32 V would make the kernel read past V's end)
    import torch
    sums = torch.zeros(3, dtype=torch.float64)
    for psi, V in ((torch.zeros(8, dtype=torch.complex128), torch.zeros(8, dtype=torch.float32)),
                   (torch.zeros(8, dtype=torch.complex64), torch.zeros(8, dtype=torch.float64)),
                   (torch.zeros(8, dtype=torch.float32), torch.zeros(8, dtype=torch.float32))):
        with pytest.raises(ValueError):
            lib.sums_noalloc(psi, V, sums)


@pytest.mark.parametrize("field,value", [("spread", 3), ("spread", -1), ("check_finite", 2), ("compensated", 2)])
def test_scheme_fields_validated(lib, field, value):
    desc = lib.make_desc(3, (16, 16, 16), (-1, -1, -1), (2, 2, 2), (0, 0, 1))
    setattr(desc, field, value)
    with pytest.raises(lib.DDIError) as e:
        lib.quadrature_tables(desc)
    assert e.value.status == -1

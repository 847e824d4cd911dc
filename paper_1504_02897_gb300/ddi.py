"""Thin ctypes binding of ``libddi_gb300.so`` (declared in ``include/ddi.h``).

Argument marshalling only: every step of the DDI / GPE path runs in the CUDA library.
Device arrays are torch tensors on the plan's device, C-contiguous, shaped
(nz, ny, nx) in 3D or (ny, nx) in 2D; real arrays are float64 (FP64 plans) or float32
(FP32 plans), complex arrays complex128 / complex64.  Loading raises if the library has
not been built (``python -c "import __graft_entry__ as g; g.build()"``): there is no
fallback.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

FP64 = 0
FP32 = 1
STOP_ENERGY = 0
STOP_PAPER = 1

_STATUS = {0: "DDI_OK", -1: "DDI_ERR_ARG", -2: "DDI_ERR_CUDA", -3: "DDI_ERR_OOM",
           -4: "DDI_ERR_NONFINITE", -5: "DDI_ERR_TIMEOUT", -6: "DDI_ERR_NOCONV", -7: "DDI_ERR_INTERNAL"}


class DDIError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {message}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("len", ctypes.c_double * 3), ("axis_n", ctypes.c_double * 3), ("axis_m", ctypes.c_double * 3),
                ("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("nphi", ctypes.c_int),
                ("kmax", ctypes.c_double), ("precision", ctypes.c_int), ("nufft_tol", ctypes.c_double),
                ("tile", ctypes.c_int * 3), ("chunk", ctypes.c_int), ("split_k0", ctypes.c_double),
                ("ellipsoid", ctypes.c_int), ("split_full_passes", ctypes.c_int), ("spread", ctypes.c_int),
                ("check_finite", ctypes.c_int), ("compensated", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("precision", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("nf", ctypes.c_int * 3), ("width", ctypes.c_int), ("beta", ctypes.c_double),
                ("nodes", ctypes.c_int64), ("nodes_used", ctypes.c_int64), ("tile", ctypes.c_int * 3),
                ("spread_items", ctypes.c_int), ("spread_split_tiles", ctypes.c_int),
                ("interp_items", ctypes.c_int), ("kmax", ctypes.c_double), ("nr", ctypes.c_int),
                ("ntheta", ctypes.c_int), ("nphi", ctypes.c_int), ("device_bytes", ctypes.c_size_t),
                ("spread_tuned_ms", ctypes.c_double), ("split_k0", ctypes.c_double), ("ellipsoid", ctypes.c_int),
                ("band", ctypes.c_int * 2), ("spread", ctypes.c_int), ("yrange", ctypes.c_int * 2)]


class GpeNonlinearity(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("damping", ctypes.c_int), ("delta", ctypes.c_double),
                ("q", ctypes.c_double)]


DAMP_NONE, DAMP_LINEAR, DAMP_POWER = 0, 1, 2


class GpeStats(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("mu", ctypes.c_double), ("Ekin", ctypes.c_double),
                ("Epot", ctypes.c_double), ("Eint", ctypes.c_double), ("Edip", ctypes.c_double),
                ("virial", ctypes.c_double), ("mass", ctypes.c_double), ("steps", ctypes.c_int),
                ("inner_max", ctypes.c_int), ("last_change", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["ddi_status_str", "ddi_last_error", "ddi_quadrature_tables", "ddi_plan_create", "ddi_plan_destroy",
           "ddi_plan_get_info", "ddi_apply", "ddi_apply_host", "ddi_apply_timed", "ddi_type2", "ddi_type1", "ddi_plan_node_order",
           "gpe_step", "gpe_energy", "gpe_ground_state", "gpe_step_adjoint", "gpe_sums_noalloc",
           "ddi_batch_create", "ddi_batch_destroy", "ddi_batch_size", "ddi_batch_get_info", "ddi_batch_apply",
           "ddi_batch_graph_stats", "ddi_plan_set_axes", "gpe_step_ex", "ddi_plan_describe", "ddi_plan_check",
           "gpe_trap_observable", "gpe_trap_gradient_workspace", "gpe_trap_gradient"]

BATCH_GRAPH = 1
BATCH_AUTOTUNE = 2
SPREAD_AUTO, SPREAD_TILES, SPREAD_COLUMNS = 0, 1, 2

_lib = None


def lib_path():
    return _build.LIB


def load():
    """Load the library (once).  Raises if it is missing: there is no CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, cd, ci = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    sig = {
        "ddi_status_str": ([ci], ctypes.c_char_p),
        "ddi_last_error": ([], ctypes.c_char_p),
        "ddi_quadrature_tables": ([ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_int64), vp, vp, vp], ci),
        "ddi_plan_create": ([ctypes.POINTER(vp), ctypes.POINTER(PlanDesc), vp], ci),
        "ddi_plan_destroy": ([vp], ci),
        "ddi_plan_get_info": ([vp, ctypes.POINTER(PlanInfo)], ci),
        "ddi_plan_describe": ([ctypes.POINTER(PlanDesc), ctypes.POINTER(PlanInfo)], ci),
        "ddi_apply": ([vp, vp, vp, vp], ci),
        "ddi_plan_check": ([vp, vp], ci),
        "ddi_apply_host": ([vp, vp, vp, vp], ci),
        "ddi_apply_timed": ([vp, vp, vp, vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(cd), ci,
                             ctypes.POINTER(ci)], ci),
        "ddi_type2": ([vp, vp, vp, vp], ci),
        "ddi_type1": ([vp, vp, vp, vp], ci),
        "ddi_plan_node_order": ([vp, vp], ci),
        "ddi_plan_set_axes": ([vp, ctypes.POINTER(cd), ctypes.POINTER(cd), vp], ci),
        "gpe_step": ([vp, vp, vp, cd, cd, cd, ci, vp], ci),
        "gpe_step_ex": ([vp, vp, vp, cd, cd, ctypes.POINTER(GpeNonlinearity), cd, ci, vp], ci),
        "gpe_energy": ([vp, vp, vp, cd, cd, ctypes.POINTER(GpeStats), vp], ci),
        "gpe_ground_state": ([vp, vp, vp, cd, cd, cd, cd, ci, cd, ci, ci, ctypes.POINTER(GpeStats), vp], ci),
        "gpe_step_adjoint": ([vp, vp, vp, vp, vp, cd, cd, cd, vp], ci),
        "gpe_sums_noalloc": ([vp, vp, ctypes.c_int64, ci, vp, vp], ci),
        "gpe_trap_observable": ([vp, vp, vp, cd, cd, cd, ci, vp, ctypes.POINTER(cd), vp], ci),
        "gpe_trap_gradient_workspace": ([vp, ci, ci, ctypes.POINTER(ctypes.c_size_t)], ci),
        "gpe_trap_gradient": ([vp, vp, vp, cd, cd, cd, ci, ci, vp, ctypes.c_size_t, ctypes.POINTER(cd), vp, vp],
                              ci),
        "ddi_batch_create": ([ctypes.POINTER(vp), ctypes.POINTER(PlanDesc), ci, ci, vp], ci),
        "ddi_batch_destroy": ([vp], ci),
        "ddi_batch_size": ([vp], ci),
        "ddi_batch_get_info": ([vp, ci, ctypes.POINTER(PlanInfo)], ci),
        "ddi_batch_apply": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], ci),
        "ddi_batch_graph_stats": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], ci),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status, where):
    if status != 0:
        msg = load().ddi_last_error().decode(errors="replace")
        raise DDIError(status, where, msg)


def make_desc(dim, n, lo, length, axis_n, axis_m=None, nr=0, ntheta=0, nphi=0, kmax=0.0,
              precision=FP64, nufft_tol=0.0, tile=None, chunk=0, split_k0=0.0, ellipsoid=False,
              split_full_passes=False, spread=0, check_finite=False, compensated=False):
    """A plan descriptor (``ddi_plan_desc``).  split_k0 != 0 selects the improved split
    algorithm of Sec. 2.1 (Eq. 3.9), 3D only: window q = exp(-|k|^2/k0^2) with k0 = split_k0
    (< 0: the library's default), the quadrature on the small ball |k| <= kmax (0: 6 k0)
    and the smooth part by a zero-padded FFT convolution.  ellipsoid: the quadrature on the
    ellipsoid |k_d| <= pi / h_d (heterogeneous boxes, e.g. thin domains h_z = eps h_x).
    split_full_passes: a split plan's ball NUFFT transforms every fine-grid line instead of
    the band around k = 0 that holds its taps (same result; for comparison).
    spread: SPREAD_AUTO (columns where they apply), SPREAD_TILES or SPREAD_COLUMNS (the
    type-1 spreading scheme, see ddi_plan_desc.spread).  check_finite: apply() synchronises
    and raises DDIError (DDI_ERR_NONFINITE) when rho holds NaN or Inf.  compensated: FP32 plans
    use Kahan sums in the column spread and head + tail twiddles in the fine-grid passes."""
    d = PlanDesc()
    d.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    lo3 = list(lo) + [0.0] * (3 - len(lo))
    ln3 = list(length) + [1.0] * (3 - len(length))
    for a in range(3):
        d.n[a] = int(nn[a])
        d.lo[a] = float(lo3[a])
        d.len[a] = float(ln3[a])
        d.axis_n[a] = float(axis_n[a])
        d.axis_m[a] = float(axis_m[a]) if axis_m is not None else 0.0
        d.tile[a] = int(tile[a]) if tile is not None else 0
    d.nr, d.ntheta, d.nphi = int(nr), int(ntheta), int(nphi)
    d.kmax = float(kmax)
    d.precision = int(precision)
    d.nufft_tol = float(nufft_tol)
    d.chunk = int(chunk)
    d.split_k0 = float(split_k0)
    d.ellipsoid = 1 if ellipsoid else 0
    d.split_full_passes = 1 if split_full_passes else 0
    d.spread = int(spread)
    d.check_finite = 1 if check_finite else 0
    d.compensated = 1 if compensated else 0
    return d


def describe(desc):
    """PlanInfo of the plan ddi_plan_create would build from desc, without building it (no GPU)."""
    info = PlanInfo()
    _check(load().ddi_plan_describe(ctypes.byref(desc), ctypes.byref(info)), "ddi_plan_describe")
    return info


def quadrature_tables(desc):
    """(k [M, dim], W [M], l0 [M, dim]) from the library's host plan builder (no GPU)."""
    lib = load()
    M = ctypes.c_int64(0)
    _check(lib.ddi_quadrature_tables(ctypes.byref(desc), ctypes.byref(M), None, None, None), "quadrature_tables")
    m = M.value
    k = np.empty((m, desc.dim), dtype=np.float64)
    W = np.empty(m, dtype=np.float64)
    l0 = np.empty((m, desc.dim), dtype=np.int32)
    _check(lib.ddi_quadrature_tables(ctypes.byref(desc), ctypes.byref(M), k.ctypes.data, W.ctypes.data,
                                     l0.ctypes.data), "quadrature_tables")
    return k, W, l0


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A DDI plan (quadrature, NUFFT tables, work lists and device workspace)."""

    def __init__(self, dim, n, lo, length, axis_n, axis_m=None, precision=FP64, stream=None, **kw):
        import torch
        lib = load()
        self.desc = make_desc(dim, n, lo, length, axis_n, axis_m, precision=precision, **kw)
        self.dim = dim
        self.precision = precision
        self.shape = tuple(reversed(list(n)[:dim]))
        self.real_dtype = torch.float64 if precision == FP64 else torch.float32
        self.cplx_dtype = torch.complex128 if precision == FP64 else torch.complex64
        h = ctypes.c_void_p()
        _check(lib.ddi_plan_create(ctypes.byref(h), ctypes.byref(self.desc), ctypes.c_void_p(_stream(stream))),
               "ddi_plan_create")
        self._h = h
        self.info = PlanInfo()
        _check(lib.ddi_plan_get_info(self._h, ctypes.byref(self.info)), "ddi_plan_get_info")
        self.dv = float(np.prod([length[d] / n[d] for d in range(dim)]))

    def set_axes(self, axis_n, axis_m=None, stream=None):
        """New dipole axes for this plan (ddi_plan_set_axes): the node weights are rebuilt
        on the device; results equal those of a plan created with these axes."""
        n = (ctypes.c_double * 3)(*[float(v) for v in axis_n])
        m = (ctypes.c_double * 3)(*[float(v) for v in axis_m]) if axis_m is not None else None
        _check(load().ddi_plan_set_axes(self._h, n, m, ctypes.c_void_p(_stream(stream))), "ddi_plan_set_axes")
        for a in range(3):
            self.desc.axis_n[a] = float(axis_n[a])
            self.desc.axis_m[a] = float(axis_m[a]) if axis_m is not None else 0.0

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ddi_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _req(self, t, complex_=False):
        dt = self.cplx_dtype if complex_ else self.real_dtype
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous() or tuple(t.shape) != self.shape:
            raise ValueError(f"expected a contiguous CUDA tensor of dtype {dt} and shape {self.shape}, got "
                             f"{t.dtype} {tuple(t.shape)} on {t.device}")
        return ctypes.c_void_p(t.data_ptr())

    def apply(self, rho, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(rho)
        _check(load().ddi_apply(self._h, self._req(rho), self._req(out), ctypes.c_void_p(_stream(stream))),
               "ddi_apply")
        return out

    def check(self, stream=None):
        """ddi_plan_check: synchronises, then raises DDIError (DDI_ERR_NONFINITE) if an
        evaluation since the last check read NaN or Inf in its rho (the record is cleared)."""
        _check(load().ddi_plan_check(self._h, ctypes.c_void_p(_stream(stream))), "ddi_plan_check")

    def apply_host(self, rho_host, out_host, stream=None):
        """End-to-end from host (numpy or pinned torch CPU) buffers; synchronises."""
        def ptr(a):
            return ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())
        _check(load().ddi_apply_host(self._h, ptr(rho_host), ptr(out_host), ctypes.c_void_p(_stream(stream))),
               "ddi_apply_host")
        return out_host

    def apply_timed(self, rho, out=None, stream=None):
        """ddi_apply with per-launch CUDA-event times: returns (out, [(kernel, ms), ...])."""
        import torch
        if out is None:
            out = torch.empty_like(rho)
        cap = 64
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = ctypes.c_int(0)
        _check(load().ddi_apply_timed(self._h, self._req(rho), self._req(out), ctypes.c_void_p(_stream(stream)),
                                      names, ms, cap, ctypes.byref(cnt)), "ddi_apply_timed")
        return out, [(names[i].decode(), ms[i]) for i in range(cnt.value)]

    def type2(self, rho, stream=None):
        import torch
        c = torch.empty(int(self.info.nodes_used), dtype=self.cplx_dtype, device=rho.device)
        _check(load().ddi_type2(self._h, self._req(rho), ctypes.c_void_p(c.data_ptr()),
                                ctypes.c_void_p(_stream(stream))), "ddi_type2")
        return c

    def type1(self, c, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=self.real_dtype, device=c.device)
        if c.dtype != self.cplx_dtype or c.numel() != int(self.info.nodes_used) or not c.is_contiguous():
            raise ValueError("c must hold nodes_used contiguous complex values of the plan precision")
        _check(load().ddi_type1(self._h, ctypes.c_void_p(c.data_ptr()), self._req(out),
                                ctypes.c_void_p(_stream(stream))), "ddi_type1")
        return out

    def node_order(self):
        q = np.empty(int(self.info.nodes_used), dtype=np.int64)
        _check(load().ddi_plan_node_order(self._h, ctypes.c_void_p(q.ctypes.data)), "ddi_plan_node_order")
        return q

    # ---- GPE ----
    def gpe_step(self, psi, V, beta, lam, dt, nsteps=1, stream=None):
        _check(load().gpe_step(self._h, self._req(psi, True), self._req(V), float(beta), float(lam), float(dt),
                               int(nsteps), ctypes.c_void_p(_stream(stream))), "gpe_step")
        return psi

    def gpe_step_ex(self, psi, V, beta, lam, dt, nsteps=1, sigma=1.0, damping=DAMP_NONE, delta=0.0, q=1.0,
                    stream=None):
        """Strang steps for the general GPE of Sec. 5 (beta |psi|^(2 sigma), damping f = 0,
        delta or delta rho^q), fixed axis; see gpe_step_ex in include/ddi.h."""
        nl = GpeNonlinearity(float(sigma), int(damping), float(delta), float(q))
        _check(load().gpe_step_ex(self._h, self._req(psi, True), self._req(V), float(beta), float(lam),
                                  ctypes.byref(nl), float(dt), int(nsteps), ctypes.c_void_p(_stream(stream))),
               "gpe_step_ex")
        return psi

    def gpe_run(self, psi, coeffs, t0, dt, nsteps, sigma=1.0, damping=DAMP_NONE, delta=0.0, q=1.0, stream=None):
        """Strang steps with time-dependent trap and coefficients (Sec. 5, e.g. the collapse
        example): coeffs(t) returns (V, beta, lambda), V a device tensor of the plan, and is
        evaluated at each step's midpoint t0 + (k + 1/2) dt; each step is one gpe_step_ex."""
        for k in range(int(nsteps)):
            V, beta, lam = coeffs(t0 + (k + 0.5) * dt)
            self.gpe_step_ex(psi, V, beta, lam, dt, 1, sigma, damping, delta, q, stream)
        return psi

    def gpe_energy(self, psi, V, beta, lam, stream=None):
        st = GpeStats()
        _check(load().gpe_energy(self._h, self._req(psi, True), self._req(V), float(beta), float(lam),
                                 ctypes.byref(st), ctypes.c_void_p(_stream(stream))), "gpe_energy")
        return st.as_dict()

    def ground_state(self, phi, V, beta, lam, dt, tol, rule=STOP_ENERGY, inner_tol=None, max_steps=100000,
                     check_every=1, stream=None):
        if inner_tol is None:
            inner_tol = 1e-13 if self.precision == FP64 else 1e-7
        st = GpeStats()
        status = load().gpe_ground_state(self._h, self._req(phi, True), self._req(V), float(beta), float(lam),
                                         float(dt), float(tol), int(rule), float(inner_tol), int(max_steps),
                                         int(check_every), ctypes.byref(st), ctypes.c_void_p(_stream(stream)))
        if status not in (0, -6):
            _check(status, "gpe_ground_state")
        out = st.as_dict()
        out["converged"] = status == 0
        return out

    def trap_observable(self, psi0, V, beta, lam, dt, nsteps, psi_T=None, stream=None):
        """J = h^d sum x_last^2 |psi_T|^2 after nsteps gpe_step steps from psi0 (gpe_trap_observable;
        psi0 is left unchanged).  Returns (J, psi_T)."""
        import torch
        if psi_T is None:
            psi_T = torch.empty_like(psi0)
        J = ctypes.c_double(0.0)
        _check(load().gpe_trap_observable(self._h, self._req(psi0, True), self._req(V), float(beta), float(lam),
                                          float(dt), int(nsteps), self._req(psi_T, True), ctypes.byref(J),
                                          ctypes.c_void_p(_stream(stream))), "gpe_trap_observable")
        return J.value, psi_T

    def trap_gradient(self, psi0, V, beta, lam, dt, nsteps, checkpoint=20, grad=None, stream=None):
        """J and dJ/dV through the hand-written adjoint with checkpointed recomputation
        (gpe_trap_gradient); the workspace is a torch buffer of the size the library asks for.
        Returns (J, grad_V)."""
        import torch
        nbytes = ctypes.c_size_t(0)
        _check(load().gpe_trap_gradient_workspace(self._h, int(nsteps), int(checkpoint), ctypes.byref(nbytes)),
               "gpe_trap_gradient_workspace")
        work = torch.empty(int(nbytes.value), dtype=torch.uint8, device=psi0.device)
        if grad is None:
            grad = torch.empty_like(V)
        J = ctypes.c_double(0.0)
        _check(load().gpe_trap_gradient(self._h, self._req(psi0, True), self._req(V), float(beta), float(lam),
                                        float(dt), int(nsteps), int(checkpoint), ctypes.c_void_p(work.data_ptr()),
                                        int(nbytes.value), ctypes.byref(J), self._req(grad),
                                        ctypes.c_void_p(_stream(stream))), "gpe_trap_gradient")
        return J.value, grad

    def step_adjoint(self, psi_in, cot, grad_V, V, beta, lam, dt, stream=None):
        _check(load().gpe_step_adjoint(self._h, self._req(psi_in, True), self._req(cot, True), self._req(grad_V),
                                       self._req(V), float(beta), float(lam), float(dt),
                                       ctypes.c_void_p(_stream(stream))), "gpe_step_adjoint")
        return cot


class Batch:
    """Many DDI evaluations in one call (ddi_batch_*): one plan per descriptor, items run
    concurrently on side streams, optionally replayed from a recorded CUDA graph, spread
    tiles optionally picked by the autotuner."""

    def __init__(self, descs, graph=True, autotune=True, stream=None):
        import torch
        lib = load()
        self.descs = list(descs)
        arr = (PlanDesc * len(self.descs))(*self.descs)
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0)
        h = ctypes.c_void_p()
        _check(lib.ddi_batch_create(ctypes.byref(h), arr, len(self.descs), flags, ctypes.c_void_p(_stream(stream))),
               "ddi_batch_create")
        self._h = h
        self.infos = []
        for i in range(len(self.descs)):
            info = PlanInfo()
            _check(lib.ddi_batch_get_info(self._h, i, ctypes.byref(info)), "ddi_batch_get_info")
            self.infos.append(info)
        self.shapes = [tuple(reversed([d.n[a] for a in range(d.dim)])) for d in self.descs]
        self.dtypes = [torch.float64 if d.precision == FP64 else torch.float32 for d in self.descs]

    def __len__(self):
        return len(self.descs)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ddi_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, rhos, outs=None, stream=None):
        import torch
        if len(rhos) != len(self):
            raise ValueError(f"expected {len(self)} densities, got {len(rhos)}")
        if outs is None:
            outs = [torch.empty_like(r) for r in rhos]
        for i, (r, o) in enumerate(zip(rhos, outs)):
            for t in (r, o):
                if (not t.is_cuda or t.dtype != self.dtypes[i] or not t.is_contiguous()
                        or tuple(t.shape) != self.shapes[i]):
                    raise ValueError(f"item {i}: expected a contiguous CUDA tensor of dtype {self.dtypes[i]} and "
                                     f"shape {self.shapes[i]}, got {t.dtype} {tuple(t.shape)} on {t.device}")
        rp = (ctypes.c_void_p * len(self))(*[r.data_ptr() for r in rhos])
        op = (ctypes.c_void_p * len(self))(*[o.data_ptr() for o in outs])
        _check(load().ddi_batch_apply(self._h, rp, op, ctypes.c_void_p(_stream(stream))), "ddi_batch_apply")
        return outs

    def graph_stats(self):
        rec, lau = ctypes.c_longlong(0), ctypes.c_longlong(0)
        _check(load().ddi_batch_graph_stats(self._h, ctypes.byref(rec), ctypes.byref(lau)), "ddi_batch_graph_stats")
        return rec.value, lau.value


def sums_noalloc(psi, V, sums, stream=None):
    """gpe_sums_noalloc: sum |psi|^2, sum V |psi|^2, sum |psi|^4 into the device tensor
    `sums` (3 float64) without any allocation by the library."""
    import torch
    # the precision follows psi; V must match it (the library reads count values of each)
    kinds = {torch.complex128: (FP64, torch.float64), torch.complex64: (FP32, torch.float32)}
    if psi.dtype not in kinds:
        raise ValueError(f"psi must be complex128 or complex64, got {psi.dtype}")
    prec, vdt = kinds[psi.dtype]
    if V.dtype != vdt:
        raise ValueError(f"V must be {vdt} for psi of dtype {psi.dtype}, got {V.dtype}")
    if not (psi.is_cuda and V.is_cuda and sums.is_cuda and psi.is_contiguous() and V.is_contiguous()
            and sums.dtype == torch.float64 and sums.numel() >= 3 and psi.numel() == V.numel()):
        raise ValueError("psi, V, sums: contiguous CUDA tensors, sums float64 with >= 3 entries")
    cur = torch.cuda.current_device()
    if not (psi.device.index == V.device.index == sums.device.index == cur):
        raise ValueError(f"psi, V and sums must be on the current device cuda:{cur}")
    _check(load().gpe_sums_noalloc(ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                   int(psi.numel()), prec, ctypes.c_void_p(sums.data_ptr()),
                                   ctypes.c_void_p(_stream(stream))), "gpe_sums_noalloc")
    return sums


def trap_gradient(plan, psi0, V, beta, lam, dt, nsteps, checkpoint=20, stream=None):
    """J = h^d sum z^2 |psi_T|^2 after nsteps TSFP steps and dJ/dV (hand-written adjoint with
    checkpointed recomputation, all in the library: gpe_trap_gradient).  Returns (J, grad_V)."""
    return plan.trap_gradient(psi0, V, beta, lam, dt, nsteps, checkpoint, stream=stream)


class TrapGradient:
    """torch.autograd.Function over the trap: forward runs the time-splitting steps and
    returns J (gpe_trap_observable); backward runs the adjoint sweep (gpe_trap_gradient, which
    recomputes the forward from checkpoints) and scales dJ/dV by the incoming gradient."""

    @staticmethod
    def apply(plan, psi0, V, beta, lam, dt, nsteps, checkpoint=20):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Vt):
                Vd = Vt.detach().contiguous()
                J, _ = plan.trap_observable(psi0, Vd, beta, lam, dt, nsteps)
                ctx.save_for_backward(Vd)
                return torch.tensor(J, dtype=torch.float64, device=Vt.device)

            @staticmethod
            def backward(ctx, gout):
                (Vd,) = ctx.saved_tensors
                _, g = plan.trap_gradient(psi0, Vd, beta, lam, dt, nsteps, checkpoint)
                return gout.to(g.dtype) * g

        return _Fn.apply(V)

"""Benchmark: 3D DDI evaluations/s at 128^3 (FP32-mixed path, error vs the FP64 path),
with the HBM roofline of the dominant kernel, an end-to-end host-buffer number and the
FP64 CPU oracle timed on this machine's cores.

Workload (one step = one DDI, i.e. one pass of the whole hot path: type-2 NUFFT (pad and
deconvolution fused into the first of 3 forward fine-grid FFT passes, interpolation at the
nodes times symbol x quadrature weights), type-1 NUFFT (spread, 3 inverse FFT passes, the
last fused with crop, deconvolution and real part)): 128^3 grid
on [-12,12)^3, density a seeded sum of 8 anisotropic Gaussians (widths U[0.5,2], centres
U[-4,4]^3), dipole axis n = (sin 30, 0, cos 30), quadrature 128 x 64 x 128 (1,048,576
nodes), NUFFT tolerance 1e-6.  Rank r of a multi-GPU run evaluates the density with seed
r (independent densities, no exchange: weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 128
L = 12.0
SIZES = dict(nr=128, ntheta=64, nphi=128)
METRIC = "3D DDI evals/s at 128^3 (FP32-mixed vs FP64, rel err <=1e-6); % of HBM roofline"
UNIT = "DDI/s"
L2_BYTES = 129 * 2 ** 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def _workload_cfg(extra=None):
    cfg = {"workload": "ddi3d_128cubed_mixture8_tilt30_quad128x64x128", "grid": [N, N, N], "box": [-L, L],
           "quadrature": [SIZES["nr"], SIZES["ntheta"], SIZES["nphi"]], "nodes": N * 64 * 128,
           "nufft_tol": 1e-6, "seed_per_rank": True, "l2": "flushed before every timed step (256 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(seconds, dist=None, device="cpu"):
    """The slowest rank's time (all ranks get it); without a process group, the local time."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(units_per_rank, world, seconds):
    """Whole-job throughput of a weak-scaling run: every rank processed units_per_rank
    independent units (its own density, seed = rank) and the job took the slowest rank's
    time."""
    return units_per_rank * world / seconds


def cpu_oracle_rate(target_s=12.0, seed=0, max_nodes=None):
    """FP64 oracle (direct nonuniform DFT) on a bounded node sample; returns DDI/s and detail.

    The oracle's cost is linear in the node count (type 2: nodes x grid, type 1: nodes x
    grid), so the time of a full DDI is the sample time scaled by M / sample nodes."""
    import numpy as np
    from oracle import nudft
    from oracle import quadrature as qd
    from paper_1504_02897_gb300 import synth
    w = synth.gaussian_mixture_density(N, L, seed=seed)
    t = qd.plan_tables(3, w["n"], w["len"], w["axis"], **SIZES)
    M = t["k"].shape[0]
    rng = np.random.default_rng(0)
    s = 512
    elapsed = 0.0
    while True:
        sel = rng.choice(M, s, replace=False)
        k, W = t["k"][sel], t["W"][sel]
        t0 = time.perf_counter()
        rh = nudft.type2(w["rho"], k, w["n"], w["lo"], w["len"])
        nudft.type1(W * rh, k, w["n"], w["lo"], w["len"])
        elapsed = time.perf_counter() - t0
        if elapsed >= target_s / 4 or (max_nodes and s >= max_nodes) or s >= M:
            break
        s = min(M, int(s * max(2.0, min(8.0, target_s / max(elapsed, 1e-3) / 2))))
    full = elapsed * M / s
    return 1.0 / full, {"sample_nodes": s, "sample_seconds": elapsed, "full_ddi_seconds_est": full}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from oracle import nudft
    from oracle import quadrature as qd
    from paper_1504_02897_gb300 import synth
    w = synth.gaussian_mixture_density(N, L, seed=0)
    t = qd.plan_tables(3, w["n"], w["len"], w["axis"], **SIZES)
    M = t["k"].shape[0]
    s = 1024
    rng = np.random.default_rng(0)
    times = []
    for it in range(args.warmup + args.steps):
        sel = rng.choice(M, s, replace=False)
        k, W = t["k"][sel], t["W"][sel]
        t0 = time.perf_counter()
        rh = nudft.type2(w["rho"], k, w["n"], w["lo"], w["len"])
        nudft.type1(W * rh, k, w["n"], w["lo"], w["len"])
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt * M / s)
    per = sum(times) / len(times)
    value = 1.0 / per
    cores = os.cpu_count()
    sample = f"{s} of {M} quadrature nodes per step (type 2 over the full 128^3 grid, type 1 onto it); " \
             f"time scaled by M/{s}"
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": _workload_cfg({"engine": "FP64 CPU oracle (direct nonuniform DFT, numpy BLAS)"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# Algorithmic bytes per launch of each kernel of the FP32 path (n = N^3 grid points,
# fine grid 2N per axis, complex 8 B): each pass moves the data it must read and write
# once; the padded / cropped passes touch only the block they need.
def fp64_path_figures(torch, stream, ms, w):
    """The FP64 path is bound by FP64 arithmetic on this part: its model FLOPs per DDI
    (interpolation 4 and spread 5 flops per tap, w^3 taps per processed node, plus the six
    fine-grid FFT passes at 5 n log2 n each) over its time, beside a probed FP64 peak
    (cuBLAS DGEMM 4096^3, best of 5)."""
    mh = N * 64 * 128 // 2
    taps = mh * w ** 3 * 9
    nf = 2 * N
    fft = 6 * 5 * nf ** 3 * math.log2(nf)
    flops = taps + fft
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(a, b)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None or t < best else best
    peak = 2 * 4096 ** 3 / (best * 1e-3) / 1e12
    del a, b
    return {"ms_per_ddi": ms, "model_gflop": flops / 1e9, "tflops": flops / (ms * 1e-3) / 1e12,
            "dgemm_probe_tflops": peak, "frac_of_probe": flops / (ms * 1e-3) / 1e12 / peak, "kernel_width": w}


def cufft_comparator(torch, stream):
    """cuFFT (through torch.fft) on the same oversampled grid, full 3D C2C forward and
    inverse of (2N)^3 complex64, best of 5: a timing comparator only (the path's own
    six passes are pruned to the padded and cropped blocks and fuse pad/crop/deconvolution)."""
    x = torch.randn(2 * N, 2 * N, 2 * N, dtype=torch.complex64, device="cuda")
    torch.fft.ifftn(torch.fft.fftn(x))
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.fft.ifftn(torch.fft.fftn(x))
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None or t < best else best
    del x
    return {"cufft_fwd_inv_ms": best, "grid": [2 * N] * 3}


def kernel_bytes(name, info, real=4):
    """Algorithmic bytes of one launch of a kernel of the 128^3 DDI: what it must read and
    write once.  The fine grid is (2N)^3 complex; the NUFFT's y passes store / read and its z
    passes transform only the fine y lines that hold node taps (info.yrange, about half);
    the spread writes those columns once; node data are the kernel values along x, y, z, the
    first taps and c_q (or the scale 2 h^d W_q) of each processed node."""
    cx = 2 * real
    n3 = N ** 3
    nf = 2 * N
    mh = int(info.nodes_used)
    w = int(info.width)
    yfrac = info.yrange[1] / nf if info.yrange[1] else 1.0
    # cells the taps reach: the ball |k| <= kmax is kmax (nf h / 2 pi) = kmax 2L / pi fine cells
    # in radius (N for the full rule, kmax = pi / h), on the k_y >= 0 side of the processed nodes
    radius = info.kmax * 2 * L / math.pi
    ball = int(4.0 / 3.0 * math.pi * (radius + w / 2.0) ** 3 * min(1.0, yfrac + w / nf)) * cx
    psi = mh * 3 * w * real + mh * 8        # kernel values and first taps
    table = {
        "pad_fft_x": n3 * real + 2 * n3 * cx,                # read rho, write N^2 rows of 2N
        "fft_y_fwd": 2 * n3 * cx + 4 * n3 * cx * yfrac,      # read the block half, write the tap lines
        "fft_z_fwd": (4 * n3 * cx + 8 * n3 * cx) * yfrac,    # the columns on the tap lines
        "interp": ball + psi + mh * real + mh * cx,          # taps' cells, node data, scale in, c_q out
        "spread": 8 * n3 * cx * yfrac + psi + mh * cx,       # tap-line columns written once, node data in
        "spread_reduce": 0,
        "fft_z_inv": (8 * n3 * cx + 4 * n3 * cx) * yfrac,
        "fft_y_inv": 4 * n3 * cx * yfrac + 2 * n3 * cx,
        "fft_x_inv_crop": 2 * n3 * cx + n3 * real,
        "fft_x_inv_crop_add": 2 * n3 * cx + 2 * n3 * real,  # also reads phi (split plans)
    }
    # the split algorithm's smooth part: the same passes without the deconvolution, every line
    smooth = {"smooth_pad_fft_x": n3 * real + 2 * n3 * cx, "smooth_fft_y_fwd": 6 * n3 * cx,
              "smooth_fft_z_symbol": 12 * n3 * cx, "smooth_fft_z_inv": 12 * n3 * cx, "smooth_fft_y_inv": 6 * n3 * cx,
              "smooth_fft_x_inv_crop": 2 * n3 * cx + n3 * real}
    return table.get(name, smooth.get(name, 0))


def profile_driver(args):
    """The 128^3 workload's DDI (8-Gaussian mixture, seed 0, on [-12,12)^3, axis (sin 30, 0,
    cos 30), quadrature 128 x 64 x 128, autotuned spread; --split: the split algorithm with the
    library's default window and ball) evaluated args.repeat times, for profilers."""
    import torch
    from paper_1504_02897_gb300 import build, ddi, synth
    build.build()
    ddi.load()
    w = synth.gaussian_mixture_density(N, L, seed=0)
    prec = ddi.FP32 if args.precision == "fp32" else ddi.FP64
    sizes = dict(split_k0=-1.0) if args.split else dict(SIZES)
    plan = ddi.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=prec, tile=(-1, 0, 0), **sizes)
    rho = torch.from_numpy(w["rho"]).to("cuda", plan.real_dtype)
    out = torch.empty_like(rho)
    for _ in range(args.repeat):
        plan.apply(rho, out)
    torch.cuda.synchronize()
    print("ok", float(out.abs().max()), "spread", "columns" if plan.info.spread == 2 else "tiles",
          list(plan.info.tile))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-split", action="store_true",
                    help="ddi3d_128: skip the split-algorithm side measurement (a child process)")
    ap.add_argument("--no-side", action="store_true",
                    help="ddi3d_128: skip the GPE and batch side measurements (child processes)")
    ap.add_argument("--workload", default="ddi3d_128",
                    choices=["ddi3d_128", "ddi3d_128_split", "batch2d_96", "tsfp128", "gs128", "grad128", "grad128_fd"],
                    help="ddi3d_128: the headline 3D workload; ddi3d_128_split: the same density by the "
                         "improved split algorithm (Eq. 3.9); batch2d_96: 96 2D densities in one batch; "
                         "tsfp128 / gs128 / grad128: the GPE step, ground state and trap gradient at 128^3")
    ap.add_argument("--fp64-check", type=int, default=1, help="grad128: also run the FP64 path for its error")
    ap.add_argument("--profile-driver", action="store_true",
                    help="no timing and no JSON: build the 128^3 workload's plan and call ddi_apply --repeat "
                         "times (the command profilers capture)")
    ap.add_argument("--repeat", type=int, default=2, help="--profile-driver: evaluations")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"], help="--profile-driver: plan precision")
    ap.add_argument("--split", action="store_true",
                    help="--profile-driver: the split algorithm's workload (library defaults for window and ball)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_driver:
        profile_driver(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch2d_96":
        bench_batch2d(args)
        return
    if args.workload == "ddi3d_128_split":
        bench_split(args)
        return
    if args.workload in ("tsfp128", "gs128", "grad128", "grad128_fd"):
        bench_gpe(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1504_02897_gb300 import build, ddi, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    ddi.load()
    dev = torch.device("cuda", torch.cuda.current_device())

    w = synth.gaussian_mixture_density(N, L, seed=rank)
    # spread tile picked by the autotuner (timed on this device, cached per shape)
    plan = ddi.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=ddi.FP32, tile=(-1, 0, 0), **SIZES)
    rho = torch.from_numpy(w["rho"]).to(dev, torch.float32)
    phi = torch.empty_like(rho)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # accuracy of the timed FP32 path against the FP64 GPU path (itself parity-tested
    # against the FP64 oracle to 1e-12)
    plan64 = ddi.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=ddi.FP64, **SIZES)
    rho64 = torch.from_numpy(w["rho"]).to(dev)
    phi64 = plan64.apply(rho64)
    plan.apply(rho, phi)
    torch.cuda.synchronize()
    err32 = float((phi.double() - phi64).abs().max() / phi64.abs().max())
    # FP64 path throughput (a few steps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    t64 = []
    for i in range(4):
        flush.fill_(float(i))
        ev[0].record(stream)
        plan64.apply(rho64, phi64)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if i > 0:
            t64.append(ev[0].elapsed_time(ev[1]))
    w64 = plan64.info.width
    del plan64, rho64, phi64
    torch.cuda.empty_cache()
    fp64 = fp64_path_figures(torch, stream, sum(t64) / len(t64), w64)
    cufft = cufft_comparator(torch, stream)

    for i in range(args.warmup):
        flush.fill_(float(i))
        plan.apply(rho, phi)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.5)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))           # L2 flush: 256 MiB write between timed steps
        starts[i].record(stream)
        plan.apply(rho, phi)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_s = sum(step_ms) / 1e3
    tmax = max_over_ranks(dev_s, dist if world > 1 else None, dev)
    value = weak_scaling_rate(args.steps, world, tmax)
    ms_per_step = tmax / args.steps * 1e3

    # per-kernel CUDA-event times (same stream, L2 flushed before each call)
    per = {}
    launches = 0
    for i in range(8):
        flush.fill_(float(i))
        _, marks = plan.apply_timed(rho, phi)
        launches = len(marks)
        if i < 2:
            continue
        for name, ms in marks:
            per.setdefault(name, []).append(ms)
    avg = {k: sum(v) / len(v) for k, v in per.items()}
    dominant = max(avg, key=avg.get)
    peaks, src = _peaks()
    peak = float(peaks["hbm_gbs"])
    info = plan.info
    alg = kernel_bytes(dominant, info)
    achieved = alg / (avg[dominant] * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic_ddi3d_128.json")
    if os.path.exists(prof):
        try:
            tr = json.load(open(prof))
            if (tr.get("kernel") == dominant and tr.get("source_hash") == _kernel_hash()
                    and tr.get("tile", list(info.tile)) == list(info.tile)):
                traffic = tr.get("bytes_per_launch")
        except Exception:
            traffic = None
    ddi_bytes = 8 * N ** 3 + 2 * 4 * (2 * N) ** 3 * 8

    # end to end: pinned host buffers, H2D + DDI + D2H inside the timed region
    host_in = torch.from_numpy(w["rho"].astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    for _ in range(2):
        plan.apply_host(host_in, host_out)
    e2e_steps = max(5, args.steps // 2)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        plan.apply_host(host_in, host_out)
    e2e_s = time.perf_counter() - t0
    e2e_value = weak_scaling_rate(e2e_steps, world, max_over_ranks(e2e_s, dist if world > 1 else None, dev))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, detail = cpu_oracle_rate()
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{detail['sample_nodes']} of {N * 64 * 128} nodes (type 2 + type 1 over the full 128^3 "
                         f"grid) in {detail['sample_seconds']:.1f} s, scaled by nodes"}

    sides = {}
    if rank == 0 and world == 1 and not args.no_split:
        sides["split_algorithm"] = split_side_run()
    if rank == 0 and world == 1 and not args.no_side:
        for wl, key in (("tsfp128", "tsfp128"), ("gs128", "gs128"), ("batch2d_96", "batch2d_96")):
            sides[key] = side_run(wl)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _workload_cfg({"fp32_rel_err_vs_fp64": err32, "fp64_ddi_per_s": 1e3 / (sum(t64) / len(t64)),
                                     "fp64_path": fp64,
                                     "nufft_points_per_s": value * 2 * N * 64 * 128,
                                     "kernel_width": info.width, "spread_tile": list(info.tile),
                                     "fft_comparator": dict(cufft, ours_six_pruned_passes_ms=sum(
                                         avg[k] for k in avg if k.startswith(("pad_", "fft_")))),
                                     "wall_s": wall}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dominant,
                         "kernel_ms": avg[dominant], "peak_source": src + " hbm_gbs (copy)"},
            "ddi_roofline": {"algorithmic_bytes": ddi_bytes, "achieved": ddi_bytes / (ms_per_step * 1e-3) / 1e9,
                             "frac": ddi_bytes / (ms_per_step * 1e-3) / 1e9 / peak, "unit": "GB/s"},
            "kernel_ms": avg,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N ** 3, "d2h_bytes_per_step": 4 * N ** 3},
            "gpu_launches": launches * args.steps,
            "clocks": clocks,
        }
        if cpu:
            out["cpu_baseline"] = cpu
        out.update(sides)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def side_run(workload, timeout_s=300):
    """Another workload measured by a child process after the headline (its own CUDA context,
    so nothing it does can touch the numbers above): the child's JSON line without the keys
    the headline already states, or the reason it has none."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", workload, "--steps", "20", "--warmup", "3",
           "--fp64-check", "1"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"error": f"no result within {timeout_s} s"}
    if r.returncode != 0:
        return {"error": f"exit status {r.returncode}: " + " | ".join(r.stderr.strip().splitlines()[-3:])}
    for line in reversed(r.stdout.strip().splitlines()):
        try:
            d = json.loads(line)
        except ValueError:
            continue
        return {k: v for k, v in d.items() if k not in ("n_gpus", "scaling", "vs_baseline", "data")}
    return {"error": "no JSON line in the child's output"}


def split_side_run(timeout_s=240):
    """The same density by the split algorithm (``--workload ddi3d_128_split``), measured by a
    child process after the headline measurement: its own CUDA context, so nothing it does
    can touch the numbers above.  Returns the child's figures, or the reason it has none."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "ddi3d_128_split", "--steps", "20",
           "--warmup", "3"]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"error": f"no result within {timeout_s} s"}
    if r.returncode != 0:
        return {"error": f"exit status {r.returncode}: " + " | ".join(r.stderr.strip().splitlines()[-3:])}
    for line in reversed(r.stdout.strip().splitlines()):
        try:
            d = json.loads(line)
        except ValueError:
            continue
        cfg = d["config"]
        return {"metric": d["metric"], "value": d["value"], "unit": d["unit"], "steps": d["steps"],
                "ms_per_step": d["ms_per_step"], "fp32_rel_err_vs_fp64": cfg["fp32_rel_err_vs_fp64"],
                "split_vs_spherical_rule_rel_diff": cfg["split_vs_spherical_rule_rel_diff"],
                "split_vs_spherical_rule_rel_diff_inner_half_box": cfg["split_vs_spherical_rule_rel_diff_inner_half_box"],
                "workload": cfg["workload"], "nodes": cfg["nodes"], "roofline": d["roofline"],
                "ddi_roofline": d["ddi_roofline"], "kernel_ms": d["kernel_ms"], "e2e": d["e2e"],
                "gpu_launches": d["gpu_launches"], "clocks": d["clocks"]}
    return {"error": "no JSON line in the child's output"}


def _timed_steps(torch, stream, flush, steps, fn):
    """Device time of `steps` calls of fn, each after a 256 MiB L2 flush, with CUDA events on
    the launching stream; nvidia-smi clocks sampled meanwhile."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.5)
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3, clocks


def bench_split(args):
    """The improved split algorithm (Sec. 2.1, Eq. 3.9) on the 128^3 mixture density of the
    headline workload: FP32 plan with the library's default window k0 = 9.6 / 24 = 0.4, ball
    |k| <= 6 k0 = 2.4 with 48 x 32 x 64 nodes, smooth part by the 2x zero-padded FFT
    convolution on the fine grid.  Reports DDI/s, the FP32 error against the FP64 split path
    (itself parity-tested against the oracle), the difference between the split result and
    the 128 x 64 x 128 spherical rule, per-kernel times and the HBM roofline of the dominant
    kernel.  One GPU (the workload is one density)."""
    import numpy as np
    import torch
    from paper_1504_02897_gb300 import build, ddi, synth

    torch.cuda.set_device(0)
    build.build()
    ddi.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    w = synth.gaussian_mixture_density(N, L, seed=0)
    plan = ddi.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=ddi.FP32, tile=(-1, 0, 0), split_k0=-1.0)
    rho = torch.from_numpy(w["rho"]).to(dev, torch.float32)
    phi = torch.empty_like(rho)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    rho64 = torch.from_numpy(w["rho"]).to(dev)
    p64 = ddi.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=ddi.FP64, split_k0=-1.0)
    phi64 = p64.apply(rho64)
    del p64
    full = ddi.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=ddi.FP64, **SIZES)
    phifull = full.apply(rho64)
    del full
    plan.apply(rho, phi)
    torch.cuda.synchronize()
    err32 = float((phi.double() - phi64).abs().max() / phi64.abs().max())
    d = (phi64 - phifull).abs()
    c = torch.arange(N, device=dev)
    inner = ((c >= N // 4) & (c < 3 * N // 4))
    m3 = inner[:, None, None] & inner[None, :, None] & inner[None, None, :]
    diff_rule = float(d.max() / phifull.abs().max())
    diff_rule_inner = float(d[m3].max() / phifull.abs().max())
    del phi64, phifull, rho64, d
    torch.cuda.empty_cache()

    for i in range(args.warmup):
        flush.fill_(float(i))
        plan.apply(rho, phi)
    dev_s, clocks = _timed_steps(torch, stream, flush, args.steps, lambda: plan.apply(rho, phi))
    value = args.steps / dev_s
    ms_per_step = dev_s / args.steps * 1e3

    per = {}
    launches = 0
    for i in range(8):
        flush.fill_(float(i))
        _, marks = plan.apply_timed(rho, phi)
        launches = len(marks)
        if i < 2:
            continue
        for name, ms in marks:
            per.setdefault(name, []).append(ms)
    avg = {k: sum(v) / len(v) for k, v in per.items()}
    dominant = max(avg, key=avg.get)
    peaks, src = _peaks()
    peak = float(peaks["hbm_gbs"])
    info = plan.info
    alg = kernel_bytes(dominant, info)
    achieved = alg / (avg[dominant] * 1e-3) / 1e9
    # the method's bytes: rho in, phi out and the smooth part's four sweeps of the padded
    # grid (write after the pad, one FFT pass, read by the crop); the ball's part is O(1) in the
    # method (here: its x passes, the spread's write of the fine grid and the band passes)
    method_bytes = 8 * N ** 3 + 4 * (2 * N) ** 3 * 8

    host_in = torch.from_numpy(w["rho"].astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    for _ in range(2):
        plan.apply_host(host_in, host_out)
    e2e_steps = max(5, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.apply_host(host_in, host_out)
    e2e_value = e2e_steps / (time.perf_counter() - t0)

    out = {
        "metric": "3D DDI evals/s at 128^3 by the split algorithm (Eq. 3.9; FP32-mixed vs FP64)", "value": value,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ddi3d_128cubed_mixture8_tilt30_split_k0_0.4_ball48x32x64", "grid": [N, N, N],
                   "box": [-L, L], "split_k0": info.split_k0, "ball_kmax": info.kmax,
                   "ball_quadrature": [info.nr, info.ntheta, info.nphi], "nodes": int(info.nodes),
                   "spread_tile": list(info.tile), "fp32_rel_err_vs_fp64": err32,
                   "split_vs_spherical_rule_rel_diff": diff_rule,
                   "split_vs_spherical_rule_rel_diff_inner_half_box": diff_rule_inner,
                   "l2": "flushed before every timed step (256 MiB write)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": dominant, "kernel_ms": avg[dominant],
                     "peak_source": src + " hbm_gbs (copy)"},
        "ddi_roofline": {"method_bytes": method_bytes,
                         "frac_of_method": method_bytes / (ms_per_step * 1e-3) / 1e9 / peak},
        "kernel_ms": avg,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N ** 3, "d2h_bytes_per_step": 4 * N ** 3},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(out))


def bench_batch2d(args):
    """96 2D densities (N in {128, 256, 512, 1024}, box length U[8, 16], tilt U[0, 90]
    degrees, 4 Gaussians each, quadrature 2N x 2N, FP32) evaluated by one ddi_batch_apply
    per step: autotuned spread tiles and one recorded CUDA graph, against the same batch
    with built-in tiles, and eager (unrecorded) launches.  Inputs (~134 MB of densities,
    ~13 GB of plan state) exceed L2; L2 is also flushed before every timed step."""
    import torch
    from paper_1504_02897_gb300 import build, ddi, synth

    torch.cuda.set_device(0)
    build.build()
    ddi.load()
    dev = torch.device("cuda", 0)
    items = synth.batch_2d(count=96, seed=0)
    descs = [ddi.make_desc(2, it["n"], it["lo"], it["len"], it["axis"], precision=ddi.FP32) for it in items]
    t0 = time.perf_counter()
    tuned = ddi.Batch(descs, graph=True, autotune=True)
    create_tuned = time.perf_counter() - t0
    t0 = time.perf_counter()
    plain = ddi.Batch(descs, graph=True, autotune=False)
    create_plain = time.perf_counter() - t0
    rhos = [torch.from_numpy(it["rho"]).to(dev, torch.float32) for it in items]
    outs = [torch.empty_like(r) for r in rhos]
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        for i in range(warmup):
            flush.fill_(float(i))
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.5)
    ms = timed(lambda: tuned.apply(rhos, outs), args.steps, args.warmup)
    clocks = sampler.stop()
    ms_plain = timed(lambda: plain.apply(rhos, outs), max(3, args.steps // 2), args.warmup)
    ms_eager = None
    eager = ddi.Batch(descs, graph=False, autotune=True)
    ms_eager = timed(lambda: eager.apply(rhos, outs), max(3, args.steps // 2), args.warmup)
    records, launches = tuned.graph_stats()

    # end to end: pinned host densities in, potentials out, inside the timed region
    host_in = [torch.from_numpy(it["rho"].astype("float32")).pin_memory() for it in items]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]

    def e2e_step():
        for h, r in zip(host_in, rhos):
            r.copy_(h, non_blocking=True)
        tuned.apply(rhos, outs)
        for o, h in zip(outs, host_out):
            h.copy_(o, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(2):
        e2e_step()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    # FP32 error of one item of each size against the FP64 path (parity-tested against the
    # oracle) applied to the same FP32-rounded density
    errs = {}
    for size in (128, 256, 512, 1024):
        i = next(j for j, it in enumerate(items) if it["n"][0] == size)
        it = items[i]
        p64 = ddi.Plan(2, it["n"], it["lo"], it["len"], it["axis"], precision=ddi.FP64)
        ref = p64.apply(rhos[i].double())
        torch.cuda.synchronize()
        errs[f"{size}^2 item {i}"] = float((outs[i].double() - ref).abs().max() / ref.abs().max())
        p64.close()
    grid_pts = sum(it["n"][0] * it["n"][1] for it in items)
    nodes = sum(int(i.nodes) for i in tuned.infos)
    # algorithmic HBM bytes of one DDI: density in and potential out (2 x 4 B per grid
    # point) and the FP32 complex fine grid (4 N^2 cells) written once by the spread and
    # read once by the first inverse FFT pass, and the same on the forward side
    ddi_bytes = sum(8 * it["n"][0] * it["n"][1] + 2 * 2 * 8 * 4 * it["n"][0] * it["n"][1] for it in items)
    peaks, src = _peaks()
    peak = float(peaks["hbm_gbs"])
    value = 96 * 1e3 / ms
    sizes = {}
    for it, inf in zip(items, tuned.infos):
        sizes.setdefault(str(it["n"][0]), list(inf.tile)[:2])
    out = {
        "metric": "2D batched DDI evals/s (96 densities, N in {128,256,512,1024}, quadrature 2N x 2N, FP32)",
        "value": value, "unit": "DDI/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batch2d_96_densities_seed0", "densities": 96, "grid_points": grid_pts,
                   "nodes": nodes, "nufft_points_per_s": value / 96 * 2 * nodes,
                   "graph": True, "autotuned_tiles": sizes, "ms_builtin_tiles": ms_plain,
                   "ms_eager_launches": ms_eager, "graph_records": records, "graph_launches": launches,
                   "create_s_autotuned": create_tuned, "create_s_builtin": create_plain,
                   "fp32_rel_err_vs_fp64_path_same_input": errs,
                   "l2": "flushed before every timed step (256 MiB write)"},
        "ddi_roofline": {"algorithmic_bytes": ddi_bytes, "achieved": ddi_bytes / (ms * 1e-3) / 1e9,
                         "peak": peak, "frac": ddi_bytes / (ms * 1e-3) / 1e9 / peak, "unit": "GB/s",
                         "peak_source": src + " hbm_gbs (copy)"},
        "e2e": {"value": 96 / e2e_s, "unit": "DDI/s", "h2d_bytes_per_step": 4 * grid_pts,
                "d2h_bytes_per_step": 4 * grid_pts},
        "clocks": clocks,
    }
    print(json.dumps(out))


def bench_gpe(args):
    """GPE workloads at 128^3 on [-10,10)^3, V = (x^2 + y^2 + 4 z^2)/2, beta = 207.16,
    lambda = 0.16 beta, dipole axis z, FP32 path (FP64 reductions), autotuned spread tile:
      tsfp128  one step = one Strang TSFP step (Eq. tssp2, Case I; dt = 1e-3), the DDI of
               |psi_1|^2 included; psi0 = the trap Gaussian with a seeded 5% perturbation
      gs128    the normalised gradient flow (backward Euler, dt = 0.01) from the trap
               Gaussian until |E^{n+1} - E^n| < 1e-10 (checked every 10 steps)
      grad128  J = h^3 sum z^2 |psi_T|^2 after 400 steps (dt = 1e-3) and dJ/dV by the
               adjoint with checkpoints every 20 steps; with --fp64-check 1 the FP64 path
               computes the same gradient for the FP32 one's error"""
    import numpy as np
    import torch
    from paper_1504_02897_gb300 import build, ddi, synth

    torch.cuda.set_device(0)
    build.build()
    ddi.load()
    dev = torch.device("cuda", 0)
    n, lo, ln = synth.box(128, 10.0, 3)
    beta, lam = 207.16, 0.16 * 207.16
    V64 = synth.harmonic_trap(n, lo, ln, (1.0, 1.0, 2.0))
    peaks, src = _peaks()
    peak = float(peaks["hbm_gbs"])

    def plan_of(prec):
        return ddi.Plan(3, n, lo, ln, (0.0, 0.0, 1.0), precision=prec, tile=(-1, 0, 0) if prec == ddi.FP32 else None)

    plan = plan_of(ddi.FP32)
    V = torch.from_numpy(V64).to(dev, torch.float32)
    sampler = ClockSampler(0)
    base = {"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic"}
    cfg = {"grid": [128, 128, 128], "box": [-10.0, 10.0], "trap": [1, 1, 2], "beta": beta, "lambda": lam,
           "axis": [0, 0, 1], "quadrature": [128, 64, 128], "spread_tile": list(plan.info.tile)}
    if args.workload == "tsfp128":
        dt = 1e-3
        psi = torch.from_numpy(synth.gpe_initial(n, lo, ln, (1.0, 1.0, 2.0), eps=0.05, seed=0)).to(dev, torch.complex64)
        m0 = plan.gpe_energy(psi, V, beta, lam)["mass"]
        for _ in range(args.warmup):
            plan.gpe_step(psi, V, beta, lam, dt, 1)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        stream = torch.cuda.current_stream()
        sampler.start()
        time.sleep(0.3)
        for i in range(args.steps):
            ev[i][0].record(stream)
            plan.gpe_step(psi, V, beta, lam, dt, 1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        m1 = plan.gpe_energy(psi, V, beta, lam)["mass"]
        step_bytes = 8 * 128 ** 3 + 2 * 4 * 256 ** 3 * 8 + 4 * 2 * 8 * 128 ** 3 + 50e6
        err = {}
        if args.fp64_check:
            # the FP32 state after 10 steps from the FP32-rounded initial state, against the FP64
            # path's 10 steps from the same rounded state (parity-tested against the oracle)
            psi0_64 = synth.gpe_initial(n, lo, ln, (1.0, 1.0, 2.0), eps=0.05, seed=0).astype(np.complex64)
            a = torch.from_numpy(psi0_64).to(dev)
            for _ in range(10):
                plan.gpe_step(a, V, beta, lam, dt, 1)
            p64 = plan_of(ddi.FP64)
            b = torch.from_numpy(psi0_64.astype(np.complex128)).to(dev)
            V64t = torch.from_numpy(V64.astype(np.float32).astype(np.float64)).to(dev)
            for _ in range(10):
                p64.gpe_step(b, V64t, beta, lam, dt, 1)
            torch.cuda.synchronize()
            err = {"fp32_rel_err_vs_fp64_10_steps": float((a.to(torch.complex128) - b).abs().max() / b.abs().max())}
            del p64
        out = dict(base, metric="TSFP steps/s at 128^3 (Eq. tssp2 Case I, DDI included, FP32-mixed)",
                   value=1e3 / ms, unit="steps/s", steps=args.steps, warmup=args.warmup, ms_per_step=ms,
                   config=dict(cfg, workload="tsfp128_dt1e-3", dt=dt, **err,
                               mass_drift_per_step=abs(m1 - m0) / (args.steps + args.warmup),
                               l2="inputs (67 MB of state) plus the 134 MB fine grid exceed L2"),
                   step_roofline={"model_bytes": step_bytes, "achieved": step_bytes / (ms * 1e-3) / 1e9,
                                  "peak": peak, "frac": step_bytes / (ms * 1e-3) / 1e9 / peak, "unit": "GB/s",
                                  "peak_source": src + " hbm_gbs (copy)"},
                   clocks=clocks)
    elif args.workload == "gs128":
        phi = torch.from_numpy(synth.gpe_initial(n, lo, ln, (1.0, 1.0, 2.0))).to(dev, torch.complex64)
        sampler.start()
        t0 = time.perf_counter()
        st = plan.ground_state(phi, V, beta, lam, 0.01, 1e-10, rule=ddi.STOP_ENERGY, max_steps=20000,
                               check_every=10)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        if args.fp64_check:
            # the FP32 path's energies of its ground state against the FP64 path's energies of
            # the same state (the FP32 state upcast)
            p64 = plan_of(ddi.FP64)
            e64 = p64.gpe_energy(phi.to(torch.complex128), torch.from_numpy(V64.astype(np.float32).astype(np.float64)).to(dev),
                                 beta, lam)
            e32 = plan.gpe_energy(phi, V, beta, lam)
            st["fp32_energy_rel_err_vs_fp64"] = {k: abs(e32[k] - e64[k]) / abs(e64[k])
                                                 for k in ("E", "mu", "Ekin", "Epot", "Eint", "Edip")}
            del p64
        out = dict(base, metric="ground state time at 128^3 (GF-BE, |dE| < 1e-10, FP32 + FP64 reductions)",
                   value=wall, unit="s", higher_is_better=False, steps=st["steps"], warmup=0,
                   ms_per_step=wall / max(1, st["steps"]) * 1e3,
                   config=dict(cfg, workload="gs128_dt0.01", dt=0.01, converged=st["converged"],
                               E=st["E"], mu=st["mu"], virial=st["virial"], mass=st["mass"],
                               last_change=st["last_change"], inner_max=st["inner_max"],
                               fp32_energy_rel_err_vs_fp64=st.get("fp32_energy_rel_err_vs_fp64")),
                   clocks=clocks)
    elif args.workload == "grad128_fd":
        # config 4's own check, in the FP64 path: dJ/dV by the adjoint (checkpoints every 20
        # steps) against central differences (J(V + eps d) - J(V - eps d)) / (2 eps), eps = 1e-4,
        # on the 16 seeded smoothed-noise directions of synth.trap_directions
        dt, nsteps, eps = 1e-3, 400, 1e-4
        del plan
        torch.cuda.empty_cache()
        p64 = plan_of(ddi.FP64)
        psi0 = torch.from_numpy(synth.gpe_initial(n, lo, ln, (1.0, 1.0, 2.0), eps=0.05, seed=0)).to(dev)
        V = torch.from_numpy(V64).to(dev)
        sampler.start()
        t0 = time.perf_counter()
        J, g = p64.trap_gradient(psi0, V, beta, lam, dt, nsteps, checkpoint=20)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - t0
        rows = []
        psiT = torch.empty_like(psi0)
        for d in synth.trap_directions(n, count=16, seed=0):
            dt_ = torch.from_numpy(d).to(dev)
            Jp, _ = p64.trap_observable(psi0, V + eps * dt_, beta, lam, dt, nsteps, psiT)
            Jm, _ = p64.trap_observable(psi0, V - eps * dt_, beta, lam, dt, nsteps, psiT)
            fd = (Jp - Jm) / (2.0 * eps)
            ad = float((g * dt_).sum().item())
            rows.append({"fd": fd, "adjoint": ad, "rel_diff": abs(fd - ad) / abs(fd)})
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        out = dict(base, metric="trap gradient vs central differences at 128^3 (FP64, 400 steps, 16 directions)",
                   value=max(r["rel_diff"] for r in rows), unit="max relative difference", higher_is_better=False,
                   dtype="f64", steps=nsteps, warmup=0, ms_per_step=t_grad / nsteps * 1e3,
                   config=dict(cfg, workload="grad128_fd_16dirs_eps1e-4", dt=dt, J=J, gradient_s=t_grad,
                               total_s=wall, directions=rows), clocks=clocks)
    else:
        dt, nsteps = 1e-3, 400
        psi0_64 = synth.gpe_initial(n, lo, ln, (1.0, 1.0, 2.0), eps=0.05, seed=0)
        psi0 = torch.from_numpy(psi0_64).to(dev, torch.complex64)
        ddi.trap_gradient(plan, psi0, V, beta, lam, dt, 20, checkpoint=20)  # warm-up
        torch.cuda.synchronize()
        sampler.start()
        t0 = time.perf_counter()
        J, g = ddi.trap_gradient(plan, psi0, V, beta, lam, dt, nsteps, checkpoint=20)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        extra = {}
        if args.fp64_check:
            del plan
            torch.cuda.empty_cache()
            p64 = plan_of(ddi.FP64)
            t1 = time.perf_counter()
            J64, g64 = ddi.trap_gradient(p64, torch.from_numpy(psi0_64).to(dev), torch.from_numpy(V64).to(dev),
                                         beta, lam, dt, nsteps, checkpoint=20)
            torch.cuda.synchronize()
            extra = {"fp64_wall_s": time.perf_counter() - t1, "J_fp64": J64,
                     "J_rel_err": abs(J - J64) / abs(J64),
                     "grad_rel_err_linf": float((g.double() - g64).abs().max() / g64.abs().max())}
        out = dict(base, metric="trap gradient time at 128^3 (400 TSFP steps + adjoint, checkpoints of 20, FP32-mixed)",
                   value=wall, unit="s", higher_is_better=False, steps=nsteps, warmup=20,
                   ms_per_step=wall / nsteps * 1e3,
                   config=dict(cfg, workload="grad128_400steps_dt1e-3", dt=dt, J=J, **extra), clocks=clocks)
    print(json.dumps(out))


def _kernel_hash():
    """Hash of the sources that determine the spread kernel's DRAM traffic: the kernel
    (nufft.cu), its work lists and node tables (plan.cu, tables.cpp/.h) and their shared
    definitions (common.cuh); the tile is checked separately.  A recorded ncu traffic
    figure is only used while these are unchanged."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1504_02897_gb300", "csrc")
    for f in ("common.cuh", "nufft.cu", "plan.cu", "tables.cpp", "tables.h"):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()

"""The multi-GPU bookkeeping of bench.py on CPU: two gloo ranks (127.0.0.1), each with its
own seeded density, agree on the slowest rank's time and the whole-job weak-scaling rate."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_1504_02897_gb300 import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        rho = synth.gaussian_mixture_density(16, 4.0, seed=rank)["rho"]   # the rank's own unit of work
        local = 1.0 + rank                                                  # rank r "took" 1 + r seconds
        tmax = bench.max_over_ranks(local, dist, "cpu")
        out.put((rank, tmax, bench.weak_scaling_rate(10, world, tmax), float(rho.sum()), float(rho[8, 8, 8])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, m0, c0), (r1, t1, v1, m1, c1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 2.0                      # both see the slowest rank
    assert v0 == v1 == pytest.approx(10 * 2 / 2.0)
    assert c0 != c1                             # different densities per rank (seed = rank)


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.weak_scaling_rate(40, 1, 0.02) == pytest.approx(2000.0)


def test_kernel_byte_model():
    # the roofline's algorithmic bytes: the split plan's smooth-part passes transform every
    # line (their NUFFT counterparts with all y lines), the accumulating crop also reads phi,
    # the z passes and the spread touch the fraction of fine y lines that hold taps, and the
    # interpolation's gathered cells follow the quadrature radius (N fine cells for the full
    # rule) on the taps' side of k_y
    sys.path.insert(0, ROOT)
    import math
    import bench

    class Info:
        nodes_used = 49152
        width = 8
        kmax = math.pi / (2 * bench.L / bench.N)
        yrange = (0, 2 * bench.N)

    n3 = bench.N ** 3
    for smooth, base in (("smooth_pad_fft_x", "pad_fft_x"), ("smooth_fft_z_symbol", "fft_z_fwd"),
                         ("smooth_fft_x_inv_crop", "fft_x_inv_crop")):
        assert bench.kernel_bytes(smooth, Info) == bench.kernel_bytes(base, Info) > 0
    assert bench.kernel_bytes("fft_x_inv_crop_add", Info) == bench.kernel_bytes("fft_x_inv_crop", Info) + 4 * n3
    node = 49152 * (3 * 8 * 4 + 8)
    full = bench.kernel_bytes("interp", Info)
    ball = int(4.0 / 3.0 * math.pi * (bench.N + 4.0) ** 3) * 8
    assert full == ball + node + 49152 * (4 + 8)
    assert bench.kernel_bytes("spread", Info) == 8 * n3 * 8 + node + 49152 * 8
    zfull = bench.kernel_bytes("fft_z_fwd", Info)
    Info.yrange = (250, bench.N + 6)          # taps on N + 6 of the 2N fine y lines
    frac = (bench.N + 6) / (2 * bench.N)
    assert bench.kernel_bytes("fft_z_fwd", Info) == pytest.approx(zfull * frac)
    assert bench.kernel_bytes("spread", Info) == pytest.approx(8 * n3 * 8 * frac + node + 49152 * 8)
    assert bench.kernel_bytes("smooth_fft_z_symbol", Info) == zfull
    Info.kmax = 2.4
    Info.yrange = (0, 2 * bench.N)
    # radius 2.4 (2L / pi) = 18.3 fine cells: the gathered ball shrinks by (22.3 / 132)^3
    assert bench.kernel_bytes("interp", Info) == int(4.0 / 3.0 * math.pi * (2.4 * 2 * bench.L / math.pi + 4.0) ** 3) * 8 \
        + node + 49152 * 12
    assert bench.kernel_bytes("no_such_kernel", Info) == 0


def test_split_side_run_reports_failure_instead_of_raising():
    # without a GPU the child process fails; the headline line then carries the reason
    sys.path.insert(0, ROOT)
    import torch
    import bench
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU")
    res = bench.split_side_run(timeout_s=300)
    assert set(res) == {"error"} and res["error"]


def test_side_run_reports_failure_instead_of_raising():
    # the GPE and batch side runs fail without a GPU; the headline line then carries the reason
    sys.path.insert(0, ROOT)
    import torch
    import bench
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU")
    res = bench.side_run("tsfp128", timeout_s=300)
    assert set(res) == {"error"} and res["error"]

"""Run the DDI on the 128^3 benchmark workload a few times (for profilers).

    python -m paper_1504_02897_gb300.drive [--precision fp32|fp64] [--repeat 3] [--n 128] [--split]

Builds the plan of bench.py's workload (8-Gaussian mixture, seed 0, on [-12,12)^3, axis
(sin 30, 0, cos 30), quadrature n x n/2 x n, autotuned spread tile) and calls ddi_apply
`repeat` times.  --split: the same density by the split algorithm with the library's
default window and ball (the ddi3d_128_split workload).
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--autotune", type=int, default=1, help="1: spread tile by the autotuner (as bench.py)")
    ap.add_argument("--tile", default="", help="fixed spread tile x,y,z (overrides --autotune)")
    ap.add_argument("--split", action="store_true", help="the split algorithm (default window and ball)")
    args = ap.parse_args()
    import torch
    from paper_1504_02897_gb300 import build, ddi, synth
    build.build()
    ddi.load()
    n = args.n
    w = synth.gaussian_mixture_density(n, 12.0, seed=0)
    prec = ddi.FP32 if args.precision == "fp32" else ddi.FP64
    sizes = dict(split_k0=-1.0) if args.split else dict(nr=n, ntheta=n // 2, nphi=n)
    plan = ddi.Plan(3, w["n"], w["lo"], w["len"], w["axis"], precision=prec,
                    tile=tuple(int(v) for v in args.tile.split(",")) if args.tile
                    else ((-1, 0, 0) if args.autotune else None), **sizes)
    rho = torch.from_numpy(w["rho"]).to("cuda", plan.real_dtype)
    out = torch.empty_like(rho)
    for _ in range(args.repeat):
        plan.apply(rho, out)
    torch.cuda.synchronize()
    print("ok", float(out.abs().max()), "tile", list(plan.info.tile))


if __name__ == "__main__":
    main()

"""Runs the path a fixed number of times on one small-to-medium workload.

A minimal driver for profiler captures (ncu) and quick timing:

    python -m paper_2511_10353_gb300.profile_case --n 512 --prec f32 --calls 1

Each call is one gg_zeldovich (positions and velocities, no displacement
output) after the plan is built, so the launch order per call is: forward z,
y, x, then for each component x inverse, y inverse, z inverse.
"""
import argparse
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_2511_10353_gb300 as gg  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--box", type=float, default=500.0)
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--calls", type=int, default=1)
    ap.add_argument("--psi", action="store_true", help="also write the displacements")
    args = ap.parse_args()
    gg.lib()
    plan = gg.Plan(args.n, args.box, gg.workloads.BBKS, 100.0, args.prec)
    shape = (args.n,) * 3
    mk = lambda: torch.empty(shape, dtype=plan.dtype, device="cuda")
    out = {"psi": [mk() for _ in range(3)] if args.psi else [None] * 3,
           "pos": [mk() for _ in range(3)], "vel": [mk() for _ in range(3)]}
    for i in range(args.calls):
        plan.zeldovich(seed=1 + i, out=out)
    plan.sync()
    torch.cuda.synchronize()
    print("ok", args.n, args.prec, args.calls)


if __name__ == "__main__":
    main()

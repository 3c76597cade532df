"""Drive the library for an external profiler (ncu): whole frames, or only the
primal-dual iterations of one level, on a seeded synthetic workload.

    python -m paper_1909_07545_gb300.profile_frame --mode frame --frames 2
    python -m paper_1909_07545_gb300.profile_frame --mode pd --level 0 --iters 100

Run from the repository root (it uses the ``synth`` scene generator).  No
CUDA graph is used, so every kernel is a separate launch a profiler can
select.  Prints the launch order of one frame so that ``ncu -s`` offsets
can be computed.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="plain_kb_1024",
                    choices=["plain_kb_1024", "plain_small_256"])
    ap.add_argument("--mode", default="frame", choices=["frame", "pd"])
    ap.add_argument("--frames", type=int, default=1)
    ap.add_argument("--level", type=int, default=0)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--block-iters", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--autotune", action="store_true",
                    help="fs_autotune the per-level schedule first (as bench.py does)")
    args = ap.parse_args()
    sys.path.insert(0, os.getcwd())
    import torch

    import synth
    from paper_1909_07545_gb300 import Solver

    pair = synth.plain_kb(args.seed) if args.workload == "plain_kb_1024" \
        else synth.plain_small(args.seed)
    H, W = pair["I0"].shape
    s = Solver(pair["cam0"], pair["cam1"], pair["R"], pair["t"], W, H, pair["levels"],
               lam=pair["lam"], huber_eps=pair["eps"], block_iters=args.block_iters)
    if args.autotune:
        print("autotuned schedule per level (0 = cluster, else blocking depth):",
              s.autotune(pair["iters"]))
    I0 = torch.as_tensor(np.float32(pair["I0"]), device="cuda")
    I1 = torch.as_tensor(np.float32(pair["I1"]), device="cuda")
    if args.mode == "frame":
        L, warps, iters = pair["levels"], pair["warps"], pair["iters"]
        for _ in range(args.frames):
            s.solve(I0, I1, warps, iters)
        torch.cuda.synchronize()
        B = args.block_iters or 4
        n = (iters + B - 1) // B
        n += n % 2
        print(f"frame: {L} levels x {warps} warps x {n} k_pd launches; k_pd launches per "
              f"level {warps * n}, before level 0: {(L - 1) * warps * n}")
    else:
        # state of a realistic warp at the chosen level, then the PD stage alone
        s.solve(I0, I1, 1, 10)
        s.stage(args.level, "TENSOR")
        s.stage(args.level, "WARP")
        torch.cuda.synchronize()
        s.stage(args.level, "PD", args.iters)
        torch.cuda.synchronize()
        print(f"pd: level {args.level} {s.level_size(args.level)}, {args.iters} iterations")
    s.close()


if __name__ == "__main__":
    main()

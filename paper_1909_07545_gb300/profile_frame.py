"""Drive the library for an external profiler (ncu): whole frames, or only the
primal-dual iterations of one level, on a seeded synthetic workload.

    python -m paper_1909_07545_gb300.profile_frame --mode frame --frames 2
    python -m paper_1909_07545_gb300.profile_frame --mode pd --level 0 --iters 100
    python -m paper_1909_07545_gb300.profile_frame --mode frame --pd-schedule persistent
    python -m paper_1909_07545_gb300.profile_frame --mode pose

Run from the repository root (it uses the ``synth`` scene generator).  No
CUDA graph is used, so every kernel is a separate launch a profiler can
select.  In frame mode one untimed frame runs first (after the autotuner,
with --autotune) and the profiled frames are bracketed by
cudaProfilerStart / Stop, so ``ncu --profile-from-start off`` captures
exactly those frames.  Pose mode brackets one fs_set_pose (the calibration
and trajectory fields) the same way.
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
    ap.add_argument("--mode", default="frame", choices=["frame", "pd", "pose"])
    ap.add_argument("--pd-schedule", default="auto", choices=["auto", "blocking", "persistent"])
    ap.add_argument("--frames", type=int, default=1)
    ap.add_argument("--level", type=int, default=0)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--block-iters", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--regularizer", default="huber_tv", choices=["huber_tv", "tgv"])
    ap.add_argument("--autotune", action="store_true",
                    help="fs_autotune the per-level schedule first (as bench.py does)")
    ap.add_argument("--schedule", default=None,
                    help="per-level schedule in fs_autotune's encoding, e.g. 7,8,15,16,16 "
                         "(the choice bench.py reports; timing-based tuning under a "
                         "profiler would see the profiler's overheads)")
    args = ap.parse_args()
    sys.path.insert(0, os.getcwd())
    import torch

    import synth
    from paper_1909_07545_gb300 import Solver

    pair = synth.plain_kb(args.seed) if args.workload == "plain_kb_1024" \
        else synth.plain_small(args.seed)
    H, W = pair["I0"].shape
    s = Solver(pair["cam0"], pair["cam1"], pair["R"], pair["t"], W, H, pair["levels"],
               lam=pair["lam"], huber_eps=pair["eps"], block_iters=args.block_iters,
               regularizer=args.regularizer, pd_schedule=args.pd_schedule)
    if args.autotune:
        print("autotuned schedule per level (0 = cluster, else blocking depth):",
              s.autotune(pair["iters"]))
    if args.schedule:
        s.set_schedule([int(v) for v in args.schedule.split(",")])
    I0 = torch.as_tensor(np.float32(pair["I0"]), device="cuda")
    I1 = torch.as_tensor(np.float32(pair["I1"]), device="cuda")
    if args.mode == "frame":
        L, warps, iters = pair["levels"], pair["warps"], pair["iters"]
        s.solve(I0, I1, warps, iters)          # warm-up frame, outside the profiled range
        torch.cuda.synchronize()
        # with ncu --profile-from-start off only these frames are captured
        torch.cuda.profiler.start()
        for _ in range(args.frames):
            s.solve(I0, I1, warps, iters)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"frame: {L} levels x {warps} warps x {iters} iterations, {args.frames} frame(s)")
    elif args.mode == "pose":
        s.set_pose(pair["R"], pair["t"])        # warm-up, outside the profiled range
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        s.set_pose(pair["R"], pair["t"])
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"pose: {W}x{H}, {pair['levels']} levels")
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

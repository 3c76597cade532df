"""Accuracy against ground truth and time per frame as functions of the warp
count N and the increment limit du_max (the trade-offs of the paper's
Sec. IV-C and V-A: Fig. 4, time linear in N while the error falls; Fig. 6,
a smaller du_max needs more warps but tracks the epipolar curve better).

    python -m paper_1909_07545_gb300.report_tradeoff [--size 800] [--levels 5]
        [--iters 10] [--scene equidistant|kb] [--deriv forward,central]
        [--precond 1] [--accel-gamma 0] [--out report.json]

Run from the repository root (it uses the ``synth`` scene generator).  The
scene is the 180-degree equidistant generator (3 textured planes at 1-5 m,
0.1 m baseline, noise-free) or the 190-degree Kannala-Brandt one (20
objects at 0.5-20 m, 0.12 m baseline, small rotation, Gaussian image noise
0.01) at the given size; --deriv lists how I_u is taken (the forward
difference of Eq. 7 and / or the central one); --precond 0 takes scalar
steps, and --accel-gamma lists gammas of the accelerated step schedule
(0 = constant steps; > 0 needs --precond 0).  Every solve is one CUDA graph replay timed
with CUDA events (mean of 3 after one untimed solve).  Errors are over the
FOV mask where the ground truth is defined: mean and median end-point error
and the fractions of pixels off by more than 1 and 5 px.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=800)
    ap.add_argument("--levels", type=int, default=5)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--warps", default="1,2,5,10,15,20")
    ap.add_argument("--du-max", default="0.1,0.2,0.5,1.0")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--scene", choices=("equidistant", "kb"), default="equidistant")
    ap.add_argument("--deriv", default="forward")
    ap.add_argument("--precond", type=int, default=1, choices=[0, 1])
    ap.add_argument("--accel-gamma", default="0")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    sys.path.insert(0, os.getcwd())
    import torch

    import synth
    from paper_1909_07545_gb300 import Solver

    W = args.size
    if args.scene == "kb":
        p = synth.plain_kb(args.seed, W=W, H=W, levels=args.levels)
    else:
        p = synth.plain_small(args.seed, W=W, H=W)
    g, valid = synth.gt_disparity(p)
    I0 = torch.as_tensor(np.float32(p["I0"]), device="cuda")
    I1 = torch.as_tensor(np.float32(p["I1"]), device="cuda")
    rows = []
    combos = [(dv, float(v), float(ga)) for dv in args.deriv.split(",")
              for v in args.du_max.split(",") for ga in args.accel_gamma.split(",")]
    for deriv, dm, ga in combos:
        s = Solver(p["cam0"], p["cam1"], p["R"], p["t"], W, W, args.levels, lam=p["lam"],
                   huber_eps=p["eps"], du_max=dm, use_graph=1, deriv=deriv,
                   precond=args.precond, accel_gamma=ga)
        s.autotune(args.iters)
        mask = s.read(0, "MASK").cpu().numpy() > 0.5
        v = valid & mask
        d = torch.empty((W, W), device="cuda")
        z = torch.empty((W, W), device="cuda")
        for n in [int(v) for v in args.warps.split(",")]:
            s.solve(I0, I1, n, args.iters, disp=d, depth=z)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                s.solve(I0, I1, n, args.iters, disp=d, depth=z)
            e1.record()
            torch.cuda.synchronize()
            err = synth.disparity_errors(d.double().cpu().numpy(), g, v)
            rows.append(dict(deriv=deriv, accel_gamma=ga, precond=args.precond, du_max=dm, warps=n, ms=e0.elapsed_time(e1) / 3, **err))
            print(json.dumps(rows[-1]), flush=True)
        s.close()
    print(f"\n{args.scene} {W}x{W}, {args.levels} levels, {args.iters} iterations per warp")
    print("| I_u | precond | gamma | du_max | N | ms/frame | EPE mean | EPE median | tau>1 | tau>5 |")
    print("|---|---:|---:|---:|---:|---:|---:|---:|---:|---:|")
    for r in rows:
        print(f"| {r['deriv']} | {r['precond']} | {r['accel_gamma']} | {r['du_max']} | {r['warps']} | "
              f"{r['ms']:.2f} | {r['epe_mean']:.3f} | "
              f"{r['epe_median']:.3f} | {100 * r['tau1']:.1f} % | {100 * r['tau5']:.1f} % |")
    if args.out:
        with open(args.out, "w") as f:
            json.dump(dict(scene=args.scene, size=W, levels=args.levels, iters=args.iters,
                           rows=rows), f, indent=1)


if __name__ == "__main__":
    main()

"""Write the oracle's disparity of the 2048 x 2048 mixed-precision workload
(synth.mixed_2048(0): the 180-degree equidistant generator, 3 planes at
1-5 m, images rounded to float32 as the GPU path receives them) at a
seeded sample of FOV pixels, at 6 levels x 2 warps x 20 iterations (a count
the oracle finishes in a few minutes), with the oracle's own response at
each sampled pixel to:

  fp32  the largest of five FP32-sized probes: (1) its pyramid images
        rounded to float32, (2) its primal-dual state rounded to float32
        after every iteration, (3) everything a float32 implementation
        stores rounded to float32, (4, 5) Gaussian relative noise of 2^-22
        and 2^-21 on both inputs;
  fp16, bf16
        what 16-bit storage rounds (float16, or bfloat16 with
        round-to-nearest-even): the level images, the tensor and step
        sizes, the linearisation I_u and rho0 once per warp and the dual p
        after every iteration, u and u_w staying exact.

Run from the repository root (a few minutes of CPU, eight processes):

    python tests/golden/make_mixed2048_oracle.py

It calls only ``oracle/`` and the input generators of ``synth/``.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "mixed2048_oracle.json")
LEVELS, WARPS, ITERS = 6, 2, 20
FP32_PROBES = ["images", "state", "all", "noise1", "noise2"]
N_SAMPLE = 8192


def _pair():
    import synth
    p = synth.mixed_2048(0)
    p["I0"] = np.float32(p["I0"]).astype(np.float64)
    p["I1"] = np.float32(p["I1"]).astype(np.float64)
    return p


def f32(a):
    return np.float32(a).astype(np.float64)


def f16(a):
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


def bf16(a):
    """float64 -> float32 -> bfloat16 (round to nearest, ties to even) -> float64."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _storage_hooks(r16):
    """Hooks that round what 16-bit storage stores (images, tensor, steps,
    linearisation, dual) with r16 and the FP32 planes with f32."""
    def images(level, a, b):
        return r16(a), r16(b)

    def on_iter(level, om, k, st, lv):
        if k == -1:
            for key in ("a", "b", "c"):
                lv[key] = r16(lv[key])
            for key in ("tau", "sig1", "sig2"):
                lv[key] = f32(lv[key])
            for key in ("Iu", "rho0"):
                st[key] = r16(st[key])
            st["u_w"] = f32(st["u_w"])
        for key in ("u", "ubar"):
            st[key] = f32(st[key])
        for key in ("p1", "p2"):
            st[key] = r16(st[key])
    return dict(level_hook=images, on_iter=on_iter)


def _solve(which):
    import oracle
    p = _pair()

    def round_state(level, om, k, st, lv):
        for key in ("u", "ubar", "p1", "p2"):
            st[key] = f32(st[key])

    def round_all(level, om, k, st, lv):
        if k == -1:
            for key in ("a", "b", "c", "tau", "sig1", "sig2"):
                lv[key] = f32(lv[key])
            for key in ("Iu", "rho0", "u_w"):
                st[key] = f32(st[key])
        round_state(level, om, k, st, lv)

    extra = {}
    if which in ("noise1", "noise2"):
        seed, rel = (12345, 2.0 ** -22) if which == "noise1" else (777, 2.0 ** -21)
        rng = np.random.default_rng(seed)
        p["I0"] = p["I0"] * (1 + rel * rng.normal(size=p["I0"].shape))
        p["I1"] = p["I1"] * (1 + rel * rng.normal(size=p["I1"].shape))
    elif which == "images":
        extra = dict(level_hook=lambda l, a, b: (f32(a), f32(b)))
    elif which == "state":
        extra = dict(on_iter=round_state)
    elif which == "all":
        extra = dict(on_iter=round_all, level_hook=lambda l, a, b: (f32(a), f32(b)))
    elif which in ("fp16", "bf16"):
        extra = _storage_hooks(f16 if which == "fp16" else bf16)
    t0 = time.time()
    ref = oracle.solve(p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"], LEVELS, WARPS,
                       ITERS, oracle.Params(lam=p["lam"], eps=p["eps"]), **extra)
    return which, ref["disp"], ref["mask"], time.time() - t0


def main():
    import synth
    jobs = ["ref"] + FP32_PROBES + ["fp16", "bf16"]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        runs = {w: (d, M, t) for w, d, M, t in pool.map(_solve, jobs)}
    d, M, secs = runs["ref"]
    ys, xs = np.nonzero(M)
    pick = np.sort(np.random.default_rng(2048).choice(len(ys), N_SAMPLE, replace=False))
    sens32 = np.max([np.abs(runs[w][0] - d) for w in FP32_PROBES], axis=0)
    s16 = {k: np.abs(runs[k][0] - d) for k in ("fp16", "bf16")}
    g, v = synth.gt_disparity(_pair())

    def field(e):
        e = e[M]
        return dict(mean=float(e.mean()), p99=float(np.quantile(e, 0.99)), max=float(e.max()),
                    n_over_5e3=int((e > 5e-3).sum()))
    out = dict(
        workload="mixed_2048(0) 2048x2048 equidistant 180 deg, 3 planes 1-5 m, "
                 f"{LEVELS} levels, {WARPS} warps x {ITERS} iterations, lam 50, eps 0.01, "
                 "images rounded to float32",
        levels=LEVELS, warps=WARPS, iters=ITERS,
        fp32_probes=FP32_PROBES,
        oracle_seconds=round(secs, 1),
        n_mask=int(M.sum()),
        disp_mean=float(d[M].mean()),
        gt_errors=synth.disparity_errors(d, g, v & M),
        probe_field=dict(fp32=field(sens32), fp16=field(s16["fp16"]), bf16=field(s16["bf16"])),
        sample_columns=["y", "x", "disp", "probe_fp32", "probe_fp16", "probe_bf16"],
        sample=[[int(ys[i]), int(xs[i]), float(d[ys[i], xs[i]]), float(sens32[ys[i], xs[i]]),
                 float(s16["fp16"][ys[i], xs[i]]), float(s16["bf16"][ys[i], xs[i]])]
                for i in pick],
    )
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {OUT}: oracle {secs:.0f} s, {out['n_mask']} FOV pixels, "
          f"probes {out['probe_field']}, gt {out['gt_errors']}")


if __name__ == "__main__":
    main()

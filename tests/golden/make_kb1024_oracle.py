"""Write the oracle's disparity of the 1024 x 1024 Kannala-Brandt workload
(synth.plain_kb(0): 5 levels, 10 warps x 100 iterations, images rounded to
float32 as the GPU path receives them) at a seeded sample of FOV pixels,
with the distribution and ground-truth error figures of the whole field.

The scene's image noise makes this solve ill-conditioned: the warps amplify
perturbations of FP32 size (Eq. 7's I_u shares its noise with rho0, so every
warp's step carries a noise-driven term).  The file therefore also holds the
oracle's own response at each sampled pixel to two such perturbations,
(1) its pyramid images rounded to float32 and (2) Gaussian relative noise of
2^-22 on both inputs, and the shift of each quantile under them.

Run from the repository root (a few minutes of CPU, three processes):

    python tests/golden/make_kb1024_oracle.py

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

OUT = os.path.join(HERE, "kb1024_oracle.json")
N_SAMPLE = 4096
QUANTILES = [0.001, 0.01, 0.1, 0.25, 0.5, 0.75, 0.9, 0.99, 0.999]


def _pair():
    import synth
    p = synth.plain_kb(0)
    p["I0"] = np.float32(p["I0"]).astype(np.float64)
    p["I1"] = np.float32(p["I1"]).astype(np.float64)
    return p


def _solve(which):
    import oracle
    p = _pair()
    extra = {}
    if which == "noise":
        rng = np.random.default_rng(12345)
        rel = 2.0 ** -22
        p["I0"] = p["I0"] * (1 + rel * rng.normal(size=p["I0"].shape))
        p["I1"] = p["I1"] * (1 + rel * rng.normal(size=p["I1"].shape))
    elif which == "images":
        f32 = lambda a: np.float32(a).astype(np.float64)
        extra = dict(level_hook=lambda l, a, b: (f32(a), f32(b)))
    t0 = time.time()
    ref = oracle.solve(p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"], p["levels"],
                       p["warps"], p["iters"], oracle.Params(lam=p["lam"], eps=p["eps"]),
                       **extra)
    return which, ref["disp"], ref["mask"], time.time() - t0


def main():
    import synth
    with mp.get_context("spawn").Pool(3) as pool:
        runs = {w: (d, M, t) for w, d, M, t in pool.map(_solve, ["ref", "images", "noise"])}
    d, M, secs = runs["ref"]
    ys, xs = np.nonzero(M)
    pick = np.sort(np.random.default_rng(1024).choice(len(ys), N_SAMPLE, replace=False))
    sens = np.maximum(np.abs(runs["images"][0] - d), np.abs(runs["noise"][0] - d))
    qref = np.quantile(d[M], QUANTILES)
    qshift = np.max([np.abs(np.quantile(runs[w][0][M], QUANTILES) - qref)
                     for w in ("images", "noise")], axis=0)
    g, v = synth.gt_disparity(_pair())
    s = sens[ys[pick], xs[pick]]
    out = dict(
        workload="plain_kb(0) 1024x1024, 5 levels, 10 warps x 100 iterations, "
                 "lam 50, eps 0.01, images rounded to float32",
        oracle_seconds=round(secs, 1),
        n_mask=int(M.sum()),
        quantile_levels=QUANTILES,
        disp_quantiles=[float(x) for x in qref],
        probe_quantile_shift=[float(x) for x in qshift],
        disp_mean=float(d[M].mean()),
        gt_errors=synth.disparity_errors(d, g, v & M),
        probe_sample_stats=dict(mean=float(s.mean()), q998=float(np.quantile(s, 0.998)),
                                max=float(s.max())),
        sample_columns=["y", "x", "disp", "probe"],
        sample=[[int(ys[i]), int(xs[i]), float(d[ys[i], xs[i]]), float(sens[ys[i], xs[i]])]
                for i in pick],
    )
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {OUT}: oracle {secs:.0f} s, {out['n_mask']} FOV pixels, "
          f"probe {out['probe_sample_stats']}, gt {out['gt_errors']}")


if __name__ == "__main__":
    main()

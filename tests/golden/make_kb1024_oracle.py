"""Write the oracle's disparity of the 1024 x 1024 Kannala-Brandt workload
(synth.plain_kb(0): 5 levels, 10 warps x 100 iterations, images rounded to
float32 as the GPU path receives them) at a seeded sample of FOV pixels,
with the distribution and ground-truth error figures of the whole field.

At this count the solve is ill-conditioned at a fraction of the pixels,
with or without image noise: ten warps per level amplify perturbations of
FP32 size where the data term has competing minima (occlusion boundaries),
and with noise also through Eq. 7's I_u, which shares its noise with rho0.
The file therefore also holds the oracle's own response at each sampled
pixel to five such perturbations -- (1) its pyramid images rounded to
float32, (2) its primal-dual state rounded to float32 after every
iteration, (3) everything a float32 implementation stores rounded to
float32, (4, 5) Gaussian relative noise of 2^-22 and 2^-21 on both inputs
-- the largest of them per pixel, and the shift of each quantile under them.

Run from the repository root (a few minutes of CPU, six processes):

    python tests/golden/make_kb1024_oracle.py            # the workload (noise 0.01)
    python tests/golden/make_kb1024_oracle.py --clean    # the same scene, noise-free

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

CLEAN = "--clean" in sys.argv
NOISE = 0.0 if CLEAN else 0.01
OUT = os.path.join(HERE, "kb1024_clean_oracle.json" if CLEAN else "kb1024_oracle.json")
PROBES = ["images", "state", "all", "noise1", "noise2"]
N_SAMPLE = 4096
QUANTILES = [0.001, 0.01, 0.1, 0.25, 0.5, 0.75, 0.9, 0.99, 0.999]


def _pair():
    import synth
    p = synth.plain_kb(0, noise=NOISE)
    p["I0"] = np.float32(p["I0"]).astype(np.float64)
    p["I1"] = np.float32(p["I1"]).astype(np.float64)
    return p


def _solve(which):
    import oracle
    p = _pair()
    f32 = lambda a: np.float32(a).astype(np.float64)
    rounded_images = lambda l, a, b: (f32(a), f32(b))

    def round_state(level, om, k, st, lv):
        for key in ("u", "ubar", "p1", "p2"):
            st[key] = f32(st[key])

    def round_all(level, om, k, st, lv):
        if k == -1:                                   # a warp's constants
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
        extra = dict(level_hook=rounded_images)
    elif which == "state":
        extra = dict(on_iter=round_state)
    elif which == "all":
        extra = dict(on_iter=round_all, level_hook=rounded_images)
    t0 = time.time()
    ref = oracle.solve(p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"], p["levels"],
                       p["warps"], p["iters"], oracle.Params(lam=p["lam"], eps=p["eps"]),
                       **extra)
    return which, ref["disp"], ref["mask"], time.time() - t0


def main():
    import synth
    with mp.get_context("spawn").Pool(len(PROBES) + 1) as pool:
        runs = {w: (d, M, t) for w, d, M, t in pool.map(_solve, ["ref"] + PROBES)}
    d, M, secs = runs["ref"]
    ys, xs = np.nonzero(M)
    pick = np.sort(np.random.default_rng(1024).choice(len(ys), N_SAMPLE, replace=False))
    sens = np.max([np.abs(runs[w][0] - d) for w in PROBES], axis=0)
    qref = np.quantile(d[M], QUANTILES)
    qshift = np.max([np.abs(np.quantile(runs[w][0][M], QUANTILES) - qref) for w in PROBES],
                    axis=0)
    g, v = synth.gt_disparity(_pair())
    s = sens[ys[pick], xs[pick]]
    out = dict(
        workload=f"plain_kb(0{', noise=0' if CLEAN else ''}) 1024x1024, 5 levels, "
                 "10 warps x 100 iterations, lam 50, eps 0.01, images rounded to float32",
        probes=PROBES,
        probe_field_stats=dict(mean=float(sens[M].mean()), max=float(sens[M].max()),
                               n_over_5e3=int((sens[M] > 5e-3).sum())),
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

"""The 2048 x 2048 mixed-precision workload (the 180-degree equidistant
generator, 6 levels, 10 warps x 100 iterations): FP32, FP16 and BF16 storage
against ground truth at the full iteration count, and against the FP64
oracle at a reduced count (6 levels x 2 warps x 20 iterations, so that the
oracle's runs stay within minutes), with the usual gates.

It renders a 2048^2 pair and runs the oracle six times (several minutes of
host time), so it runs only when FS_REPORT=1; FS_REPORT_OUT names a file for
the JSON report."""
import json
import os

import numpy as np
import pytest

import synth
from gpu_helpers import (disparity_parity, f32pair, make_solver, np64, oracle_sensitivity,
                         oracle_solve)

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("FS_REPORT") != "1",
                                 reason="report run: set FS_REPORT=1")]

REDUCED = dict(warps=2, iters=20)


def _round(kind):
    import torch
    dt = {"f16": torch.float16, "bf16": torch.bfloat16}[kind]
    return lambda a: torch.as_tensor(a, dtype=torch.float32).to(dt).to(torch.float64).numpy()


def _timed_solve(s, I0, I1, warps, iters, reps=3):
    import torch
    d, z = s.solve(I0, I1, warps, iters)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        d, z = s.solve(I0, I1, warps, iters, disp=d, depth=z)
    e1.record()
    torch.cuda.synchronize()
    return d, e0.elapsed_time(e1) / reps


def test_mixed_precision_2048_against_oracle_and_ground_truth():
    from paper_1909_07545_gb300 import build
    build.build()
    p = f32pair(synth.mixed_2048(0))
    g, v = synth.gt_disparity(p)
    report = {"workload": "equidistant 180 deg, 2048x2048, 3 planes 1-5 m, 6 levels",
              "full": {}, "reduced_vs_oracle": {}}

    ref = oracle_solve(p, **REDUCED)
    M = ref["mask"]
    v = v & M
    report["oracle_reduced_vs_gt"] = synth.disparity_errors(ref["disp"], g, v)
    sens = oracle_sensitivity(p, ref, **REDUCED)
    probes = {k: oracle_solve(p, level_hook=(lambda r: lambda l, a, b: (r(a), r(b)))(_round(k)),
                              **REDUCED)["disp"] for k in ("f16", "bf16")}

    failures = []
    for kind in ("f32", "f16", "bf16"):
        s = make_solver(p, storage=kind, use_graph=1)
        s.autotune(p["iters"])
        d, ms = _timed_solve(s, p["I0"], p["I1"], p["warps"], p["iters"])
        report["full"][kind] = dict(ms_per_frame=ms, **synth.disparity_errors(np64(d), g, v))
        dr, _ = _timed_solve(s, p["I0"], p["I1"], REDUCED["warps"], REDUCED["iters"], reps=1)
        dr = np64(dr)
        err = np.abs(dr - ref["disp"])[M]
        row = dict(mean=float(err.mean()), p99=float(np.quantile(err, 0.99)),
                   max=float(err.max()))
        if kind == "f32":
            ok, rep = disparity_parity(dr, ref, sens)
            row["gate"] = rep
            if not ok:
                failures.append((kind, rep))
        else:
            pe = np.abs(probes[kind] - ref["disp"])[M]
            row.update(probe_mean=float(pe.mean()), probe_p99=float(np.quantile(pe, 0.99)))
            if not (row["mean"] <= 3 * row["probe_mean"] and row["p99"] <= 3 * row["probe_p99"]):
                failures.append((kind, row))
        report["reduced_vs_oracle"][kind] = row
        s.close()
    print(json.dumps(report))
    out = os.environ.get("FS_REPORT_OUT")
    if out:
        with open(out, "w") as f:
            json.dump(report, f, indent=1)
    assert not failures, failures

"""End-to-end GPU solve (fs_solve through the C ABI) against the FP64 oracle.

Same float32 inputs, pyramid, warp and iteration counts on both sides.  The
disparity gate (gpu_helpers.disparity_parity): mean |dd| <= 1e-4 px over the
FOV mask, max |dd| <= 5e-3 px over the pixels the oracle's own FP32-sized
probes leave within 1e-3 px, and the ill-conditioned rest no worse than the
oracle's own response to those probes.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import (disparity_parity, f32pair, make_solver, np64, oracle_params,
                         oracle_sensitivity, ragged_pair)

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_07545_gb300 import build
    build.build()


def _oracle(pair, levels=None, warps=None, iters=None, d_init=None, w_init=None, **prm):
    return oracle.solve(pair["I0"], pair["I1"], pair["cam0"], pair["cam1"], pair["R"],
                        pair["t"], levels or pair["levels"], warps or pair["warps"],
                        iters or pair["iters"], oracle_params(pair, **prm), d_init=d_init,
                        w_init=w_init)


def _compare(pair, ref, disp, depth, sens):
    M = ref["mask"]
    d = np64(disp)
    assert np.all(d[~M] == 0.0)
    ok, rep = disparity_parity(d, ref, sens)
    assert ok, rep
    z = np64(depth)
    assert np.all(np.isnan(z[~M]))
    # range follows the disparity: compare where the oracle is stable and the
    # warp is at least a pixel long
    w = np.linalg.norm(ref["w"], axis=-1)
    sel = M & (w > 1.0) & (sens <= 1e-4) & np.isfinite(ref["depth"]) & (ref["depth"] > 0)
    rel = np.abs(z[sel] / ref["depth"][sel] - 1.0)
    assert np.median(rel) < 1e-4
    assert rel.max() < 1e-2
    return rep


@pytest.fixture(scope="module")
def small():
    return f32pair(synth.plain_small(0))


@pytest.fixture(scope="module")
def small_ref(small):
    ref = _oracle(small)
    return ref, oracle_sensitivity(small, ref)


def test_plain_small_256_matches_oracle(small, small_ref):
    s = make_solver(small)
    disp, depth = s.solve(small["I0"], small["I1"], small["warps"], small["iters"])
    _compare(small, small_ref[0], disp, depth, small_ref[1])
    s.close()


@pytest.mark.parametrize("models", [("ucm", "ucm"), ("eucm", "ucm")])
def test_unified_model_pairs_match_oracle(models):
    # the unified and enhanced unified lenses (Sec. III-B, III-D), camera 1
    # possibly of the other model (the calibration field then also carries
    # the difference of the lenses, Sec. IV-A)
    from gpu_helpers import unified_pair
    p = unified_pair(11, model0=models[0], model1=models[1])
    ref = _oracle(p)
    sens = oracle_sensitivity(p, ref)
    s = make_solver(p)
    disp, depth = s.solve(p["I0"], p["I1"], p["warps"], p["iters"])
    _compare(p, ref, disp, depth, sens)
    s.close()


def test_tiny_odd_sized_pair_matches_oracle():
    # 37 x 29: a single partial tile per level, ragged on both axes
    p = f32pair(synth.plain_small(6, W=37, H=29))
    ref = _oracle(p, levels=2, warps=3, iters=25)
    sens = oracle_sensitivity(p, ref, levels=2, warps=3, iters=25)
    s = make_solver(p, levels=2)
    disp, depth = s.solve(p["I0"], p["I1"], 3, 25)
    d = np64(disp)
    assert np.all(d[~ref["mask"]] == 0.0)
    ok, rep = disparity_parity(d, ref, sens)     # disparities here are below a pixel
    assert ok, rep
    s.close()


def test_tgv_solve_matches_oracle(small):
    # the paper's own regulariser, TGV-L1 (Eq. 10-11), through the whole
    # method: 3 levels x 3 warps x 30 iterations
    ref = _oracle(small, warps=3, iters=30, regularizer="tgv")
    sens = oracle_sensitivity(small, ref, warps=3, iters=30, regularizer="tgv")
    s = make_solver(small, regularizer="tgv", use_graph=1)
    choice = s.autotune(8)             # launch per step (0) or blocking on a footprint
    assert len(choice) == small["levels"] and all(0 <= c <= 40 for c in choice)
    disp, depth = s.solve(small["I0"], small["I1"], 3, 30)
    _compare(small, ref, disp, depth, sens)
    s.close()


@pytest.mark.parametrize("block", [1, 5, 8])
def test_schedules_and_block_depths_are_identical(small, block):
    s1 = make_solver(small, block_iters=block, pd_schedule=1)
    s0 = make_solver(small)
    d1, z1 = s1.solve(small["I0"], small["I1"], 2, 13)
    d0, z0 = s0.solve(small["I0"], small["I1"], 2, 13)
    assert np.array_equal(np64(d1), np64(d0))
    s1.close()
    s0.close()


def test_ragged_rotated_pair_matches_oracle():
    pair = ragged_pair(1)
    ref = _oracle(pair)
    sens = oracle_sensitivity(pair, ref)
    s = make_solver(pair)
    disp, depth = s.solve(pair["I0"], pair["I1"], pair["warps"], pair["iters"])
    _compare(pair, ref, disp, depth, sens)
    s.close()


def test_central_derivative_matches_oracle():
    # I_u as the central difference along the trajectory (the option beside
    # Eq. 7's forward difference) on the noisy Kannala-Brandt rig at 256^2
    p = f32pair(synth.plain_kb(0, W=256, H=256, levels=3))
    ref = _oracle(p, warps=5, iters=50, deriv="central")
    sens = oracle_sensitivity(p, ref, warps=5, iters=50, deriv="central")
    s = make_solver(p, deriv="central")
    disp, depth = s.solve(p["I0"], p["I1"], 5, 50)
    _compare(p, ref, disp, depth, sens)
    s.close()


@pytest.mark.parametrize("gamma", [0.05, 0.5])
def test_accelerated_schedule_matches_oracle(small, gamma):
    # Chambolle-Pock Algorithm 2 steps (accel_gamma), restarted every warp
    ref = _oracle(small, warps=3, iters=40, precond=False, accel_gamma=gamma)
    sens = oracle_sensitivity(small, ref, warps=3, iters=40, precond=False, accel_gamma=gamma)
    s = make_solver(small, precond=0, accel_gamma=gamma)
    disp, depth = s.solve(small["I0"], small["I1"], 3, 40)
    _compare(small, ref, disp, depth, sens)
    d0 = np64(disp)
    s.close()
    # every schedule gives the same bits: blocking depths, footprints, the
    # tuner, graph replay (iteration k of a warp reads entry k of the table
    # whichever launch it falls in)
    for prm in (dict(pd_schedule=1, block_iters=1), dict(pd_schedule=1, block_iters=7),
                dict(use_graph=1)):
        t = make_solver(small, precond=0, accel_gamma=gamma, **prm)
        if prm.get("use_graph"):
            choice = t.autotune(40)
            assert all(c >= 1 for c in choice)          # no cluster schedule here
            t.solve(small["I0"], small["I1"], 3, 40)
        d, _ = t.solve(small["I0"], small["I1"], 3, 40)
        assert np.array_equal(np64(d), d0), prm
        t.close()


def test_unpreconditioned_steps_match_oracle(small):
    ref = _oracle(small, warps=3, iters=40, precond=False)
    sens = oracle_sensitivity(small, ref, warps=3, iters=40, precond=False)
    s = make_solver(small, precond=0)
    disp, depth = s.solve(small["I0"], small["I1"], 3, 40)
    _compare(small, ref, disp, depth, sens)
    s.close()


def test_graph_replay_and_host_entry_point(small, small_ref):
    s = make_solver(small, use_graph=1)
    import torch
    I0 = torch.as_tensor(np.float32(small["I0"]), device="cuda")
    I1 = torch.as_tensor(np.float32(small["I1"]), device="cuda")
    outs = []
    for _ in range(3):
        d, z = s.solve(I0, I1, small["warps"], small["iters"])
        outs.append(np64(d))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    _compare(small, small_ref[0], d, z, small_ref[1])
    hd, hz = s.solve_host(small["I0"], small["I1"], small["warps"], small["iters"])
    assert np.array_equal(hd.astype(np.float64), outs[0])
    s.close()


def test_full_size_kb_1024_short_schedule():
    # the full 1024 x 1024 Kannala-Brandt workload (5 levels) on a schedule the
    # oracle finishes in seconds: 2 warps x 20 iterations per level
    pair = f32pair(synth.plain_kb(0))
    ref = _oracle(pair, warps=2, iters=20)
    sens = oracle_sensitivity(pair, ref, warps=2, iters=20)
    s = make_solver(pair)
    disp, depth = s.solve(pair["I0"], pair["I1"], 2, 20)
    _compare(pair, ref, disp, depth, sens)
    s.close()


def test_warm_start_matches_oracle(small):
    # warm start from a disparity (here the oracle's own cold result, rounded
    # to float32): w rebuilt along the trajectory field, finest level only
    cold = _oracle(small, warps=2, iters=20)
    d0 = np.float32(cold["disp"]).astype(np.float64)
    ref = _oracle(small, warps=3, iters=30, d_init=d0)
    sens = oracle_sensitivity(small, ref, warps=3, iters=30, d_init=d0)
    s = make_solver(small)
    disp, depth = s.solve(small["I0"], small["I1"], 3, 30, init=d0)
    _compare(small, ref, disp, depth, sens)
    # the rebuilt warp vector itself, before any iteration
    s.solve(small["I0"], small["I1"], 1, 1, init=d0)
    s.close()


def test_continue_matches_oracle(small):
    # continuation of a video stream: the finest level's u and w (here the
    # oracle's cold result, rounded to float32, written into the handle) are
    # taken as they are; finest level only
    import paper_1909_07545_gb300 as fsb
    s = make_solver(small)
    with pytest.raises(fsb.FsError):          # nothing to continue from yet
        s.solve_continue(small["I0"], small["I1"], 1, 1)
    cold = _oracle(small, warps=2, iters=20)
    d0 = np.float32(cold["disp"]).astype(np.float64)
    w0 = np.float32(cold["w"]).astype(np.float64)
    ref = _oracle(small, warps=3, iters=30, d_init=d0, w_init=w0)
    sens = oracle_sensitivity(small, ref, warps=3, iters=30, d_init=d0, w_init=w0)
    s.solve(small["I0"], small["I1"], 1, 2)   # any result, then replaced
    s.write(0, "U", d0)
    s.write(0, "W", np.moveaxis(w0, -1, 0))
    disp, depth = s.solve_continue(small["I0"], small["I1"], 3, 30)
    _compare(small, ref, disp, depth, sens)
    s.autotune(iters=4)                       # overwrites the state
    with pytest.raises(fsb.FsError):
        s.solve_continue(small["I0"], small["I1"], 1, 1)
    s.close()


def test_batch_results_equal_lone_solves(small):
    # pairs of three sizes (256^2, ragged 203x157, 128^2) solved concurrently
    # through one batch graph: each result is bit-identical to its lone solve
    import paper_1909_07545_gb300 as fsb
    pairs = [small, ragged_pair(2), f32pair(synth.plain_small(3, W=128, H=128))]
    for p in pairs[1:]:
        p.setdefault("warps", 3)
    alone = []
    for p in pairs:
        s = make_solver(p)
        d, z = s.solve(p["I0"], p["I1"], 3, 25)
        alone.append((np64(d), np64(z)))
        s.close()
    solvers = [make_solver(p) for p in pairs]
    batch = fsb.Batch(solvers)
    # no bound, then one and two pairs at a time on the finest level
    for limit in (0, 1, 2):
        batch.set_finest_limit(limit)
        for rep in range(2):                 # capture, then replay
            ds, zs = batch.solve([p["I0"] for p in pairs], [p["I1"] for p in pairs], 3, 25)
            for (d, z), (ad, az) in zip(zip(ds, zs), alone):
                assert np.array_equal(np64(d), ad)
                assert np.array_equal(np64(z), az, equal_nan=True)
    with pytest.raises(fsb.FsError):
        batch.set_finest_limit(-1)
    # the coarse levels' common schedule tuned for the batch: same bits
    c = batch.autotune(iters=10)
    assert c in (-1, 32, 69, 8, 45)
    ds, zs = batch.solve([p["I0"] for p in pairs], [p["I1"] for p in pairs], 3, 25)
    for (d, z), (ad, az) in zip(zip(ds, zs), alone):
        assert np.array_equal(np64(d), ad)
        assert np.array_equal(np64(z), az, equal_nan=True)
    with pytest.raises(fsb.FsError):
        batch.autotune(iters=0)
    batch.close()
    for s in solvers:
        s.close()


def test_autotuned_schedule_gives_identical_results(small):
    s0 = make_solver(small)
    d0, _ = s0.solve(small["I0"], small["I1"], 2, 13)
    s1 = make_solver(small)
    choice = s1.autotune(iters=12)
    assert len(choice) == small["levels"] and all(0 <= c <= 71 for c in choice)
    d1, _ = s1.solve(small["I0"], small["I1"], 2, 13)
    assert np.array_equal(np64(d0), np64(d1))
    s0.close()
    s1.close()


def test_set_pose_equals_a_handle_created_with_that_pose():
    # a per-frame pose change recomputes the calibration field (Sec. IV-A) and
    # the trajectory fields (Sec. III-B) in place; the result is the same as
    # a handle created with the new pose, also through a captured graph
    p = ragged_pair(3)
    R, t = p["R"], p["t"]
    s1 = make_solver(p, use_graph=1)
    s1.set_pose(np.eye(3), np.array([-0.08, 0.0, 0.01]))
    s1.solve(p["I0"], p["I1"], 2, 10)              # captures a graph with that pose
    s1.set_pose(R, t)
    s2 = make_solver(p, use_graph=1)
    for l in range(p["levels"]):
        assert np.array_equal(np64(s1.trajectory_field(l)), np64(s2.trajectory_field(l)))
    d1, z1 = s1.solve(p["I0"], p["I1"], 2, 10)
    d2, z2 = s2.solve(p["I0"], p["I1"], 2, 10)
    assert np.array_equal(np64(s1.read(0, "I1")), np64(s2.read(0, "I1")))
    assert np.array_equal(np64(d1), np64(d2))
    assert np.array_equal(np64(z1), np64(z2), equal_nan=True)
    s1.close()
    s2.close()


def test_set_schedule_reproduces_a_tuned_schedule(small):
    import paper_1909_07545_gb300 as fsb
    s1 = make_solver(small)
    choice = s1.autotune(iters=6)
    s2 = make_solver(small)
    s2.set_schedule(choice)
    d1, _ = s1.solve(small["I0"], small["I1"], 2, 11)
    d2, _ = s2.solve(small["I0"], small["I1"], 2, 11)
    assert np.array_equal(np64(d1), np64(d2))
    s2.set_schedule([28, 36, 45])              # every level on an explicit schedule
    d3, _ = s2.solve(small["I0"], small["I1"], 2, 11)
    assert np.array_equal(np64(d1), np64(d3))
    with pytest.raises(fsb.FsError):
        s2.set_schedule([72, -1, -1])
    s1.close()
    s2.close()


def test_degenerate_constant_images_give_zero_disparity(small):
    # no texture: I_u = 0 everywhere, the data term has no slope, so every
    # step leaves u at 0 (and the range is +inf where the rays coincide)
    p = dict(small, I0=np.full_like(small["I0"], 0.5), I1=np.full_like(small["I1"], 0.5))
    s = make_solver(p)
    disp, depth = s.solve(p["I0"], p["I1"], 2, 10)
    d, z = np64(disp), np64(depth)
    M = np64(s.read(0, "MASK")) > 0.5
    assert np.all(d == 0.0)
    assert np.all(np.isposinf(z[M])) and np.all(np.isnan(z[~M]))
    s.close()


def test_large_frame_properties():
    # 4096 x 4096, 7 levels (beyond what the oracle can solve here): outputs
    # finite inside the FOV, zero / NaN outside, and two schedules identical
    import math
    W = 4096
    rng = np.random.default_rng(9)
    yy, xx = np.mgrid[0:W, 0:W].astype(np.float32)
    img = 0.5 + 0.2 * np.sin(xx / 17.0) * np.cos(yy / 23.0) + 0.05 * rng.random((W, W))
    cam = dict(model="equidistant", fx=1280.0, fy=1280.0, cx=(W - 1) / 2, cy=(W - 1) / 2,
               k=[0, 0, 0, 0], fov_deg=180.0)
    pair = dict(I0=img, I1=np.roll(img, -3, axis=1), cam0=cam, cam1=dict(cam), R=np.eye(3),
                t=np.array([-0.1, 0.0, 0.0]), levels=7, lam=50.0, eps=0.01)
    outs = []
    for sched in (None, [16] * 7):
        s = make_solver(pair, use_graph=1)
        if sched:
            s.set_schedule(sched)
        d, z = s.solve(pair["I0"], pair["I1"], 1, 6)
        M = np64(s.read(0, "MASK")) > 0.5
        outs.append((np64(d), np64(z)))
        s.close()
    d, z = outs[0]
    assert np.all(np.isfinite(d[M])) and np.all(d[~M] == 0.0) and np.all(np.isnan(z[~M]))
    assert np.abs(d[M]).max() < 0.2 * 1 * (2 ** 7 - 1) + 1e-3    # reach of 1 warp per level
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1], equal_nan=True)
    assert math.isfinite(float(d[M].mean()))


@pytest.mark.parametrize("fixture", ["kb1024_oracle.json", "kb1024_clean_oracle.json"])
def test_bench_configuration_at_full_counts(fixture):
    # the timed configuration itself: 1024^2 Kannala-Brandt, 5 levels x 10
    # warps x 100 iterations, autotuned schedule in a CUDA graph, on the
    # workload's noisy scene and on the same scene without noise, against
    # the oracle's disparity at 4096 seeded FOV pixels and its quantiles
    # (tests/golden/*.json, written by make_kb1024_oracle.py).
    # At ten warps per level the solve is chaotic at a fraction of the
    # pixels, noise or not: the FP64 oracle itself moves there by up to a few
    # pixels under FP32-sized perturbations (the five probes of the
    # fixture), mostly at occlusion boundaries, so the stated per-pixel
    # bound cannot hold for any FP32 implementation at this count.  The gate
    # compares distributions with the oracle's own: mean, 99.8th percentile
    # and maximum of |dd| at the sampled pixels no more than twice the
    # probes' (floors 1e-4 / 5e-3 / 5e-3 px), no more sampled pixels above
    # 5e-3 px than twice the probes' count + 4, and the quantiles of the
    # field within twice their probe shift (floor 2e-3 px); on the noise-free
    # scene also max |dd| <= 5e-3 px at the samples no probe moves by more
    # than 1e-3 px.  What holds at
    # any size: the same bits as the default schedule, zero / NaN off the
    # FOV, the reach of the clipped increments.
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", fixture)) as f:
        gold = json.load(f)
    p = f32pair(synth.plain_kb(0, noise=0.0 if "clean" in fixture else 0.01))
    outs = []
    for tuned in (True, False):
        s = make_solver(p, use_graph=1)
        if tuned:
            s.autotune(p["iters"])
        d, z = s.solve(p["I0"], p["I1"], p["warps"], p["iters"])
        d, z = s.solve(p["I0"], p["I1"], p["warps"], p["iters"], disp=d, depth=z)   # replay
        M = np64(s.read(0, "MASK")) > 0.5
        outs.append((np64(d), np64(z)))
        s.close()
    (d, z), (d0, z0) = outs
    assert np.array_equal(d, d0) and np.array_equal(z, z0, equal_nan=True)
    assert int(M.sum()) == gold["n_mask"]
    assert np.all(d[~M] == 0.0) and np.all(np.isnan(z[~M]))
    assert np.abs(d[M]).max() <= 0.2 * p["warps"] * (2 ** p["levels"] - 1) + 1e-3
    ys, xs, dref, probe = (np.array(c) for c in zip(*gold["sample"]))
    err = np.abs(d[ys.astype(int), xs.astype(int)] - dref)
    ps = gold["probe_sample_stats"]
    well = probe <= 1e-3
    rep = dict(mean=err.mean(), q998=float(np.quantile(err, 0.998)), max=err.max(),
               n_over=int((err > 5e-3).sum()), n_over_probe=int((probe > 5e-3).sum()),
               n_well=int(well.sum()), max_well=float(err[well].max()), probe=ps)
    print(fixture, rep)
    assert rep["mean"] <= max(1e-4, 2 * ps["mean"]), rep
    assert rep["q998"] <= max(5e-3, 2 * ps["q998"]), rep
    assert rep["max"] <= max(5e-3, 2 * ps["max"]), rep
    assert rep["n_over"] <= 2 * rep["n_over_probe"] + 4, rep
    if "clean" in fixture:
        # without image noise, the stated bound holds at full count on the
        # samples that no probe moves by more than 1e-3 px
        assert rep["max_well"] <= 5e-3, rep
    qs = np.quantile(d[M], gold["quantile_levels"])
    tol = np.maximum(2e-3, 2 * np.array(gold["probe_quantile_shift"]))
    assert np.all(np.abs(qs - gold["disp_quantiles"]) <= tol), (qs, gold["disp_quantiles"], tol)

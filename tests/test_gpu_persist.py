"""The persistent schedule (pd_schedule = FS_SCHED_PERSISTENT): every level
and warp of a cold solve -- or of a batch of pairs of uneven sizes -- in one
persistent launch over a device work list, each tile waiting on its
neighbours' counters.  It runs the same per-pixel functions as the
launch-per-stage schedule, so its results are the same bits; every wait is
bounded and a wait that runs out ends the launch with FS_ETIMEOUT."""
import numpy as np
import pytest

import synth
from gpu_helpers import f32pair, make_solver, np64, ragged_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_07545_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def small():
    return f32pair(synth.plain_small(0))


def _solve(pair, warps, iters, levels=None, tune=0, **prm):
    s = make_solver(pair, levels=levels, **prm)
    if tune:
        s.autotune(tune)
    d, z = s.solve(pair["I0"], pair["I1"], warps, iters)
    d, z = np64(d), np64(z)
    s.close()
    return d, z


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1], equal_nan=True)


@pytest.mark.parametrize("case", ["small", "ragged", "tiny", "kb1024"])
def test_persistent_solve_is_bit_identical(case, small):
    pair, levels, warps, iters = {
        "small": (small, 3, 3, 25),
        "ragged": (ragged_pair(1), 3, 3, 17),
        "tiny": (f32pair(synth.plain_small(6, W=37, H=29)), 2, 2, 9),
        "kb1024": (f32pair(synth.plain_kb(0)), 5, 2, 20),
    }[case]
    ref = _solve(pair, warps, iters, levels)
    for graph in (0, 1):
        got = _solve(pair, warps, iters, levels, pd_schedule="persistent", use_graph=graph)
        _same(got, ref)


@pytest.mark.parametrize("prm", [dict(storage="f16"), dict(storage="bf16"),
                                 dict(deriv="central"), dict(precond=0),
                                 dict(block_iters=3)])
def test_persistent_options_are_bit_identical(small, prm):
    # with 16-bit storage the dual is rounded to storage at every block
    # boundary, so the reference is the blocking schedule with the same depth
    # (in FP32 every schedule gives the same bits)
    prm = dict(prm)
    if "storage" in prm:
        prm["block_iters"] = 5
    ref = _solve(small, 2, 14, pd_schedule="blocking", **prm)
    got = _solve(small, 2, 14, pd_schedule="persistent", use_graph=1, **prm)
    _same(got, ref)


@pytest.mark.parametrize("iters", [1, 2, 7])
def test_persistent_iteration_counts(small, iters):
    # one iteration: two blocks per warp, the second copying the state across
    ref = _solve(small, 2, iters)
    _same(_solve(small, 2, iters, pd_schedule="persistent"), ref)


def test_persistent_tuned_geometry_is_bit_identical(small):
    # footprints and depths from fs_autotune's choices (the 32-wide choices
    # and depths 9..15 included)
    ref = _solve(small, 2, 30)
    got = _solve(small, 2, 30, tune=30, pd_schedule="persistent", use_graph=1)
    _same(got, ref)
    s = make_solver(small, pd_schedule="persistent")
    s.set_schedule([31, 52, 44])
    d, z = s.solve(small["I0"], small["I1"], 2, 30)
    _same((np64(d), np64(z)), ref)
    s.close()


def test_persistent_batch_of_uneven_pairs_equals_lone_solves():
    # pairs of four sizes and two level counts in one persistent launch, FP16
    # storage, each result the same bits as its lone launch-per-stage solve
    # with the same blocking depth
    import paper_1909_07545_gb300 as fsb
    pairs = [f32pair(synth.plain_small(0)), ragged_pair(2),
             f32pair(synth.plain_kb(4, W=160, H=144, levels=2)),
             f32pair(synth.plain_small(3, W=96, H=112))]
    levels = [3, 3, 2, 2]
    alone = [_solve(p, 2, 12, levels=L, storage="f16", pd_schedule="blocking", block_iters=6)
             for p, L in zip(pairs, levels)]
    solvers = [make_solver(p, levels=L, storage="f16", pd_schedule="persistent", block_iters=6)
               for p, L in zip(pairs, levels)]
    batch = fsb.Batch(solvers)
    for rep in range(2):                       # capture, then replay
        ds, zs = batch.solve([p["I0"] for p in pairs], [p["I1"] for p in pairs], 2, 12)
        for d, z, a in zip(ds, zs, alone):
            _same((np64(d), np64(z)), a)
    batch.close()
    for s in solvers:
        s.close()


def test_persistent_wait_runs_out_with_timeout_status(small):
    # a wait on a counter nothing advances gives up after the limit: the
    # solve returns FS_ETIMEOUT, the context stays usable, and the next
    # solve (without the stall) gives the usual bits
    import time

    import paper_1909_07545_gb300 as fsb
    ref = _solve(small, 2, 10)
    for graph in (0, 1):
        s = make_solver(small, pd_schedule="persistent", use_graph=graph)
        s.set_wait_limit(0.05)
        s.persist_stall(True)
        t0 = time.perf_counter()
        with pytest.raises(fsb.FsError) as err:
            s.solve(small["I0"], small["I1"], 2, 10)
        assert err.value.status == -5                     # FS_ETIMEOUT
        assert time.perf_counter() - t0 < 5.0
        s.persist_stall(False)
        d, z = s.solve(small["I0"], small["I1"], 2, 10)
        _same((np64(d), np64(z)), ref)
        s.close()
    with pytest.raises(fsb.FsError):
        make_solver(small).set_wait_limit(0.0)


def test_persistent_batch_wait_runs_out(small):
    import paper_1909_07545_gb300 as fsb
    pairs = [small, ragged_pair(2)]
    solvers = [make_solver(p, pd_schedule="persistent") for p in pairs]
    for s in solvers:
        s.set_wait_limit(0.05)
    solvers[1].persist_stall(True)
    batch = fsb.Batch(solvers)
    with pytest.raises(fsb.FsError) as err:
        batch.solve([p["I0"] for p in pairs], [p["I1"] for p in pairs], 2, 8)
    assert err.value.status == -5
    solvers[1].persist_stall(False)
    batch.solve([p["I0"] for p in pairs], [p["I1"] for p in pairs], 2, 8)
    batch.close()
    for s in solvers:
        s.close()


def test_persistent_handle_warm_start_uses_blocking(small):
    # warm starts and continuations of a persistent handle take the
    # launch-per-stage path: the same bits as a default handle
    d0 = np.float32(_solve(small, 2, 10)[0]).astype(np.float64)
    ref_s = make_solver(small)
    ref = ref_s.solve(small["I0"], small["I1"], 2, 10, init=d0)
    ref = (np64(ref[0]), np64(ref[1]))
    ref_c = ref_s.solve_continue(small["I0"], small["I1"], 2, 10)
    ref_c = (np64(ref_c[0]), np64(ref_c[1]))
    s = make_solver(small, pd_schedule="persistent")
    got = s.solve(small["I0"], small["I1"], 2, 10, init=d0)
    _same((np64(got[0]), np64(got[1])), ref)
    got = s.solve_continue(small["I0"], small["I1"], 2, 10)
    _same((np64(got[0]), np64(got[1])), ref_c)
    s.close()
    ref_s.close()


def test_persistent_deep_halo_repeats_bit_for_bit():
    # the bench configuration at full count with a tuned schedule whose
    # coarsest level runs depth 12 on 32 x 32 footprints: an 8-pixel
    # interior under a 12-pixel halo, so each footprint reaches two tiles to
    # every side and its items wait on 25 tiles.  Four solves in a row, each
    # the same bits as the launch-per-stage schedule.
    import torch
    pair = f32pair(synth.plain_kb(0))
    tuned = [31, 32, 48, 49, 52]
    ref = make_solver(pair, use_graph=1)
    ref.set_schedule(tuned)
    d0, _ = ref.solve(pair["I0"], pair["I1"], 10, 100)
    d0 = d0.clone()
    ref.close()
    s = make_solver(pair, use_graph=1, pd_schedule="persistent")
    s.set_schedule(tuned)
    for _ in range(4):
        d, _ = s.solve(pair["I0"], pair["I1"], 10, 100)
        assert torch.equal(d, d0)
    s.close()

"""The TMA-staged primal-dual footprints (fs_autotune choices 56..63,
k_pd_tma.cu): 64 x 64 footprints laid out 48 columns apart, inputs copied
into shared memory by the tensor memory accelerator while a resident CTA
iterates on the previous footprint.  The interior of a footprint after
n <= B iterations depends only on its dependency cone, so every footprint
geometry gives the same bits as the launch-per-footprint kernel (whose
results the oracle comparisons pin).  With 16-bit storage the dual is
rounded at every launch boundary, so equal bits need equal depths.

The 1024 x 1024 level has 462 footprints at depth 7, three or four per
resident CTA, so these cases run the prefetch of the next footprint; the
small and ragged levels have one per CTA and exercise the edges (zero fill
of copies that reach outside the level)."""
import time

import numpy as np
import pytest

import synth
from gpu_helpers import f32pair, make_solver, np64, ragged_pair

pytestmark = pytest.mark.gpu

TMA = 55            # choice TMA + d = depth d on the TMA footprints
T1024 = 24          # choice T1024 + d = depth d on 64 x 64 footprints of 1024 threads


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_07545_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def kb():
    return f32pair(synth.plain_kb(0))


@pytest.fixture(scope="module")
def small():
    return f32pair(synth.plain_small(0))


def _run(pair, sched, warps, iters, levels=None, **prm):
    s = make_solver(pair, levels=levels, **prm)
    s.set_schedule(sched)
    d, z = s.solve(pair["I0"], pair["I1"], warps, iters)
    out = (np64(d), np64(z), np64(s.read(0, "P")))
    s.check_waits()
    s.close()
    return out


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1], equal_nan=True)
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("depth", [6, 7, 8])
def test_tma_footprints_match_k_pd_on_the_1024_frame(kb, depth):
    # 5 levels x 2 warps x 20 iterations; the two finest levels on the TMA
    # footprints against the same depths on k_pd's 64 x 64 footprints
    rest = [-1, -1, -1]
    ref = _run(kb, [T1024 + depth, T1024 + min(depth, 8)] + rest, 2, 20)
    got = _run(kb, [TMA + depth, TMA + min(depth, 8)] + rest, 2, 20)
    _same(got, ref)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_tma_footprints_match_k_pd_with_16_bit_storage(kb, storage):
    ref = _run(kb, [T1024 + 7, T1024 + 8, -1, -1, -1], 2, 20, storage=storage)
    got = _run(kb, [TMA + 7, TMA + 8, -1, -1, -1], 2, 20, storage=storage)
    _same(got, ref)


def test_tma_footprints_every_depth_on_the_small_levels(small):
    # the 256 x 256 workload (3 levels), every level on the TMA footprints
    ref = _run(small, [-1, -1, -1], 2, 17)
    for depth in range(1, 9):
        _same(_run(small, [TMA + depth] * 3, 2, 17), ref)


def test_tma_footprints_on_a_ragged_level():
    # 203 x 157 with an off-centre principal point: footprints cut by the
    # right and bottom edges at every depth
    pair = ragged_pair(0)
    ref = _run(pair, [-1, -1, -1], 2, 13)
    for depth in (1, 3, 5, 8):
        _same(_run(pair, [TMA + depth, TMA + depth, -1], 2, 13), ref)


def test_tma_footprints_with_the_accelerated_schedule(small):
    prm = dict(accel_gamma=0.35, precond=0)
    ref = _run(small, [T1024 + 6, -1, -1], 2, 15, **prm)
    got = _run(small, [TMA + 6, -1, -1], 2, 15, **prm)
    _same(got, ref)


def test_tma_footprints_in_a_graph_and_a_batch(kb):
    import paper_1909_07545_gb300 as fsb
    sched = [TMA + 7, TMA + 8, -1, -1, -1]
    ref = _run(kb, sched, 2, 20)
    s = make_solver(kb, use_graph=1)
    s.set_schedule(sched)
    for _ in range(2):                           # capture, then replay
        d, z = s.solve(kb["I0"], kb["I1"], 2, 20)
        _same((np64(d), np64(z), np64(s.read(0, "P"))), ref)
    s.close()
    pairs = [kb, f32pair(synth.plain_kb(1))]
    solvers = []
    for p in pairs:
        t = make_solver(p)
        t.set_schedule(sched)
        solvers.append(t)
    b = fsb.Batch(solvers)
    ds, zs = b.solve([p["I0"] for p in pairs], [p["I1"] for p in pairs], 2, 20)
    assert np.array_equal(np64(ds[0]), ref[0])
    alone = _run(pairs[1], sched, 2, 20)
    assert np.array_equal(np64(ds[1]), alone[0])
    b.close()
    for t in solvers:
        t.check_waits()
        t.close()


def test_tma_footprints_are_tried_by_the_autotuner(small):
    s = make_solver(small)
    choice = s.autotune(iters=6)
    assert all(-1 <= c <= 71 for c in choice)
    s.close()


def test_tma_wait_runs_out_with_timeout_status(small):
    # the first launch of each TMA level waits for 16 bytes no copy delivers:
    # every CTA gives up after the limit, fs_check_waits reports FS_ETIMEOUT
    # once, the context stays usable and the next solve gives the usual bits
    import paper_1909_07545_gb300 as fsb
    sched = [TMA + 6, -1, -1]
    ref = _run(small, sched, 2, 10)
    s = make_solver(small)
    s.set_schedule(sched)
    s.set_wait_limit(0.05)
    s.persist_stall(True)
    t0 = time.perf_counter()
    s.solve(small["I0"], small["I1"], 2, 10)
    with pytest.raises(fsb.FsError) as err:
        s.check_waits()
    assert err.value.status == -5                     # FS_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    s.check_waits()                                   # the record was cleared
    s.persist_stall(False)
    d, z = s.solve(small["I0"], small["I1"], 2, 10)
    s.check_waits()
    _same((np64(d), np64(z), np64(s.read(0, "P"))), ref)
    # fs_solve_host checks by itself
    s.persist_stall(True)
    with pytest.raises(fsb.FsError) as err:
        s.solve_host(small["I0"], small["I1"], 2, 10)
    assert err.value.status == -5
    s.persist_stall(False)
    s.close()

"""Guard-band mode (FS_GUARD_BANDS=1): the out-of-bounds check that stands in
for a memory sanitizer.  Every device plane of a handle sits between bands of
0xFF bytes; fs_guard_check (run after every solve in this mode) reports a band
that a kernel stored into, and a kernel that loaded from a band would read NaN
or all mask bits and change its results.  So each configuration below is
solved with and without bands and must give the same bits, with every band
intact: the schedules (cluster, temporal blocking on each footprint, depths
1..8), the storage types, TGV, warm start, continuation, batches, pose
changes, odd and tiny sizes.  A clobbered band must be reported.
"""
import os

import numpy as np
import pytest

import synth
from synth.render import rotation
from gpu_helpers import f32pair, make_solver, np64, ragged_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_07545_gb300 import build
    build.build()


class _Guard:
    def __enter__(self):
        self.old = os.environ.get("FS_GUARD_BANDS")
        os.environ["FS_GUARD_BANDS"] = "1"

    def __exit__(self, *exc):
        if self.old is None:
            os.environ.pop("FS_GUARD_BANDS", None)
        else:
            os.environ["FS_GUARD_BANDS"] = self.old


def _run(pair, guarded, levels=None, prep=None, solve=None, **prm):
    if guarded:
        with _Guard():
            s = make_solver(pair, levels=levels, **prm)
        assert s.guard_clobber() > 0
    else:
        s = make_solver(pair, levels=levels, **prm)
    if prep is not None:
        prep(s)
    out = solve(s) if solve is not None else s.solve(pair["I0"], pair["I1"], 2, 17)
    res = [np64(t) for t in out]
    if guarded:
        s.guard_check()
    s.close()
    return res


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)


@pytest.fixture(scope="module")
def small():
    return f32pair(synth.plain_small(0))


@pytest.mark.parametrize("prm", [
    dict(),                                             # automatic: cluster + blocking
    dict(pd_schedule=1, block_iters=1),
    dict(pd_schedule=1, block_iters=8),
    dict(use_graph=1),
    dict(storage="f16"),
    dict(storage="bf16"),
    dict(deriv="central"),
    dict(regularizer="tgv", block_iters=4),
    dict(regularizer="tgv", block_iters=1),
])
def test_guarded_solves_match_unguarded(small, prm):
    _same(_run(small, True, **prm), _run(small, False, **prm))


@pytest.mark.parametrize("choice", [1, 5, 8, 9, 12, 16, 17, 20, 24, 25, 29, 32, 33, 37, 40,
                                    41, 45, 48, 49, 55, 56, 60, 63, 64, 69])
def test_guarded_footprints_and_depths(small, choice):
    # every temporal-blocking footprint (64x64 of 512 and of 1024 threads; 32x32
    # of 256, 512 and 1024 threads; 64x32; the TMA-staged 64x64; 64x48 of 768
    # threads) at several depths
    sched = lambda s: s.set_schedule([choice] * small["levels"])
    _same(_run(small, True, prep=sched), _run(small, False, prep=sched))


def test_guarded_tgv_per_step_schedule(small):
    sched = lambda s: s.set_schedule([0] * small["levels"])
    _same(_run(small, True, prep=sched, regularizer="tgv"),
          _run(small, False, prep=sched, regularizer="tgv"))


@pytest.mark.parametrize("size", [(37, 29), (203, 157), (130, 66)])
def test_guarded_odd_sizes(size):
    W, H = size
    p = ragged_pair(3, W=W, H=H) if W > 100 and H > 100 else f32pair(
        synth.plain_small(4, W=W, H=H))
    _same(_run(p, True, levels=2), _run(p, False, levels=2))


def test_guarded_warm_start_continue_and_pose(small):
    def seq(s):
        d, z = s.solve(small["I0"], small["I1"], 2, 15)
        d1, z1 = s.solve(small["I0"], small["I1"], 2, 15, init=d)       # warm start
        d2, z2 = s.solve_continue(small["I0"], small["I1"], 1, 15)
        R = rotation([0.3, 1.0, 0.1], np.radians(0.7))
        s.set_pose(R, small["t"])
        d3, z3 = s.solve(small["I0"], small["I1"], 2, 15)
        s.energy(0)
        return d, z, d1, z1, d2, z2, d3, z3
    _same(_run(small, True, solve=seq), _run(small, False, solve=seq))


def test_guarded_batch(small):
    import paper_1909_07545_gb300 as fsb
    other = f32pair(synth.plain_small(1))
    res = []
    for guarded in (True, False):
        if guarded:
            with _Guard():
                ss = [make_solver(small), make_solver(other)]
        else:
            ss = [make_solver(small), make_solver(other)]
        b = fsb.Batch(ss, finest_limit=1)
        out = b.solve([small["I0"], other["I0"]], [small["I1"], other["I1"]], 2, 15)
        res.append([np64(t) for pair in out for t in pair])
        if guarded:
            for s in ss:
                s.guard_check()
        b.close()
        for s in ss:
            s.close()
    _same(res[0], res[1])


def test_autotune_under_guard_bands(small):
    # every candidate of the tuner (cluster, each footprint and depth) runs
    with _Guard():
        s = make_solver(small, use_graph=1)
    s.autotune(20)
    s.guard_check()
    s.close()


def test_clobbered_band_is_reported(small):
    import paper_1909_07545_gb300 as fsb
    with _Guard():
        s = make_solver(small)
    n = s.guard_clobber()
    # before each plane, the calibration field and the status word, and the end
    assert n == small["levels"] * 25 + 3
    s.guard_check()
    s.guard_clobber(band=5, offset=100)            # the band before level 0's u_w plane
    with pytest.raises(fsb.FsError, match="level 0 u_w"):
        s.guard_check()
    with pytest.raises(fsb.FsError):
        s.guard_clobber(band=n)
    s.close()
    t = make_solver(small)                          # made without bands
    with pytest.raises(fsb.FsError, match="FS_GUARD_BANDS"):
        t.guard_check()
    t.close()

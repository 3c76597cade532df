"""Failure handling under host-side fault injection: FS_FAULT_ALLOC makes the
library's device allocation at a named site fail (cudaErrorMemoryAllocation,
without reaching the device).  Each call must return FS_ENOMEM with a
message, leak nothing that a later call trips over, and work again once the
fault is gone; a server request whose rig cannot be made resident fails alone
while the other rigs' requests complete.  No GPU fault is involved.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import f32pair, make_solver, np64

pytestmark = pytest.mark.gpu

ENOMEM = -2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_07545_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def small():
    return f32pair(synth.plain_small(0, W=128, H=128))


def _raises_enomem(fn):
    import paper_1909_07545_gb300 as fsb
    with pytest.raises(fsb.FsError) as e:
        fn()
    assert e.value.status == ENOMEM, e.value
    return e.value


def test_create_fails_cleanly_and_recovers(small, monkeypatch):
    monkeypatch.setenv("FS_FAULT_ALLOC", "arena")
    for _ in range(3):                                   # repeated failures leak nothing
        _raises_enomem(lambda: make_solver(small, levels=3))
    monkeypatch.setenv("FS_GUARD_BANDS", "1")
    monkeypatch.setenv("FS_FAULT_ALLOC", "guard")        # the second allocation of a create
    _raises_enomem(lambda: make_solver(small, levels=3))
    monkeypatch.delenv("FS_GUARD_BANDS")
    monkeypatch.delenv("FS_FAULT_ALLOC")
    s = make_solver(small, levels=3)
    d, _ = s.solve(small["I0"], small["I1"], 2, 10)
    assert np.isfinite(np64(d)).all()
    s.close()


def test_lazy_allocations_fail_then_succeed(small, monkeypatch):
    # the staging planes of the host entry point, the energy accumulators and
    # the accelerated schedule's table are allocated on first use
    s = make_solver(small, levels=3)
    ref, _ = s.solve(small["I0"], small["I1"], 2, 10)
    ref = np64(ref)
    monkeypatch.setenv("FS_FAULT_ALLOC", "stage")
    _raises_enomem(lambda: s.solve_host(small["I0"], small["I1"], 2, 10))
    monkeypatch.setenv("FS_FAULT_ALLOC", "energy")
    _raises_enomem(lambda: s.energy(0))
    monkeypatch.delenv("FS_FAULT_ALLOC")
    d, _ = s.solve_host(small["I0"], small["I1"], 2, 10)
    assert np.array_equal(np.asarray(d, dtype=np.float64), ref)
    assert np.isfinite(s.energy(0)[0])
    s.close()
    a = make_solver(small, levels=3, precond=0, accel_gamma=0.1)
    monkeypatch.setenv("FS_FAULT_ALLOC", "sched")
    _raises_enomem(lambda: a.solve(small["I0"], small["I1"], 2, 10))
    monkeypatch.delenv("FS_FAULT_ALLOC")
    d, _ = a.solve(small["I0"], small["I1"], 2, 10)
    assert np.isfinite(np64(d)).all()
    a.close()


def test_server_request_fails_alone(monkeypatch):
    import paper_1909_07545_gb300 as fsb
    rigs = []
    for seed, W in ((0, 96), (1, 112)):
        q = synth.rig_sequence(seed, W, W, n_frames=2)
        q["frames"] = [(np.ascontiguousarray(np.float32(a)), np.ascontiguousarray(np.float32(b)))
                       for a, b, _ in q["frames"]]
        rigs.append(q)
    srv = fsb.Server(warps=2, iters=10, cold_warps=2, cold_iters=10, max_inflight=2)
    ids = [srv.add_rig(q["cam0"], q["cam1"], q["R"], q["t"], q["frames"][0][0].shape[1],
                       q["frames"][0][0].shape[0], q["levels"], lam=q["lam"], huber_eps=q["eps"])
           for q in rigs]
    # rig 0's first request: its state cannot be allocated
    monkeypatch.setenv("FS_FAULT_ALLOC", "planes")
    r0 = srv.submit(ids[0], *rigs[0]["frames"][0])
    with pytest.raises(fsb.FsError) as e:
        srv.wait(r0)
    assert e.value.status == ENOMEM
    monkeypatch.delenv("FS_FAULT_ALLOC")
    # the other rig, and then rig 0 itself, are served
    srv.wait(srv.submit(ids[1], *rigs[1]["frames"][0]))
    srv.wait(srv.submit(ids[0], *rigs[0]["frames"][0]))
    srv.wait(srv.submit(ids[0], *rigs[0]["frames"][1]))
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 4      # completed counts the failed one
    srv.close()

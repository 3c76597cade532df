"""The serving leg's load generator (bench.serve_leg) against a stand-in
server on the CPU: every request is submitted once and waited for exactly
once, each rig's result buffers come back through that rig's own waiter,
Python's collector is running again afterwards, and the line carries the
server's figures beside the generator's own lateness."""
import gc
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _StandInServer:
    """The calls serve_leg makes on fs_server, with the server's ordering:
    a rig's requests run one after another (0.3 ms each here), rigs run side
    by side, and a request may be waited for once only."""

    def __init__(self, fail_every=0, **cfg):
        self.fail_every = fail_every
        self.cfg = cfg
        self.mu = threading.Condition()
        self.next_id = 0
        self.rig_of, self.done, self.waited = {}, {}, set()
        self.lat, self.rig_queues = [], []
        self.t_first = self.t_last = None
        self.closed = False

    def add_rig(self, cam0, cam1, R, t, W, H, levels, **prm):
        q = []
        self.rig_queues.append(q)
        return len(self.rig_queues) - 1

    def _run(self, rid, t0):
        time.sleep(0.0003)
        with self.mu:
            self.done[rid] = True
            self.lat.append(1e3 * (time.perf_counter() - t0))
            self.t_last = time.perf_counter()
            self.mu.notify_all()

    def submit(self, rig, I0, I1, disp, depth):
        assert not self.closed
        assert I0.shape == I1.shape == disp.shape == depth.shape
        with self.mu:
            self.next_id += 1
            rid = self.next_id
            self.rig_of[rid] = rig
            if self.t_first is None:
                self.t_first = time.perf_counter()
            prev = self.rig_queues[rig][-1] if self.rig_queues[rig] else None
            self.rig_queues[rig].append(rid)
        t0 = time.perf_counter()

        def after_previous():
            if prev is not None:                 # a rig's requests in order
                with self.mu:
                    self.mu.wait_for(lambda: prev in self.done)
            self._run(rid, t0)

        threading.Thread(target=after_previous, daemon=True).start()
        return rid

    def wait(self, rid):
        with self.mu:
            assert rid in self.rig_of and rid not in self.waited, rid
            self.waited.add(rid)
            self.mu.wait_for(lambda: rid in self.done)
        if self.fail_every and rid % self.fail_every == 0:
            raise RuntimeError(f"request {rid} failed")
        return 0.0

    def drain(self):
        with self.mu:
            self.mu.wait_for(lambda: len(self.done) == self.next_id)

    def stats(self, reset=False):
        with self.mu:
            v = np.sort(np.array(self.lat)) if self.lat else np.zeros(1)
            span = (self.t_last - self.t_first) if self.t_first else 0.0
            out = dict(completed=len(self.lat), failed=0, cold=0, evictions=0,
                       resident_bytes=0, p50_ms=float(np.percentile(v, 50)),
                       p99_ms=float(np.percentile(v, 99)), max_ms=float(v[-1]),
                       mean_ms=float(v.mean()),
                       frames_per_s=len(self.lat) / span if span > 0 else 0.0)
            if reset:
                self.lat, self.t_first = [], None
            return out

    def close(self):
        self.closed = True


@pytest.mark.parametrize("fail_every", [0, 7])
def test_generator_waits_each_request_once_per_rig(monkeypatch, fail_every):
    # fail_every = 7: every seventh request fails when it is waited for; its
    # rig's buffer still comes back and the run completes
    import bench
    import paper_1909_07545_gb300 as pkg
    made = []

    def server(**cfg):
        made.append(_StandInServer(fail_every=fail_every, **cfg))
        return made[-1]

    monkeypatch.setattr(pkg, "Server", server)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    W, n_rigs = 16, 5
    frame = (np.zeros((W, W)), np.zeros((W, W)), None)
    rigs = [dict(cam0={}, cam1={}, R=np.eye(3), t=np.zeros(3), levels=2, lam=50.0, eps=0.01,
                 frames=[frame] * 3) for _ in range(n_rigs)]
    assert gc.isenabled()
    out = bench.serve_leg(rigs, [W] * n_rigs, 0, 0.5, 300.0, 2, 1)
    assert gc.isenabled()                     # the collector runs again afterwards
    srv = made[0]
    assert srv.closed
    # warm-up (3 per rig), the open loop, and 64 per rig saturated: every
    # request waited for exactly once
    assert srv.next_id == 3 * n_rigs + out["requests"] + 64 * n_rigs
    assert srv.waited == set(srv.rig_of)
    assert 100 < out["requests"] < 220        # 0.5 s of Poisson arrivals at 300/s
    assert out["failed"] == 0 and out["saturated_requests"] == 64 * n_rigs
    late = out["submit_late_ms"]
    assert set(late) == {"p50", "p99", "max"}
    assert 0.0 <= late["p50"] <= late["p99"] <= late["max"]
    for key in ("p50_ms", "p99_ms", "max_ms", "frames_per_s", "submit_stalls",
                "saturated_frames_per_s", "workload"):
        assert key in out

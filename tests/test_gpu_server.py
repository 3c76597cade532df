"""fs_server: requests from several rigs served concurrently give the same
bits as the same requests served alone and as a lone handle's solve chain;
admission by memory budget evicts idle rigs (which then restart cold); the
16-bit served path stays within the storage's accuracy of the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import np64, oracle_solve

pytestmark = pytest.mark.gpu

COLD = (3, 20)      # warps x iterations per level, first frame of a rig
WARM = (2, 15)      # warps x iterations on the finest level, later frames


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_07545_gb300 import build
    build.build()


def _f32(a):
    return np.ascontiguousarray(np.float32(a))


@pytest.fixture(scope="module")
def rigs():
    # three rigs of different sizes and calibrations, three frames each
    out = []
    for seed, (W, H) in [(0, (128, 128)), (1, (112, 96)), (2, (160, 144))]:
        q = synth.rig_sequence(seed, W, H, n_frames=3)
        q["frames"] = [(_f32(a), _f32(b), g) for a, b, g in q["frames"]]
        out.append(q)
    return out


def _server(**kw):
    import paper_1909_07545_gb300 as fsb
    cfg = dict(warps=WARM[0], iters=WARM[1], cold_warps=COLD[0], cold_iters=COLD[1])
    cfg.update(kw)
    return fsb.Server(**cfg)


def _add(srv, q, **prm):
    H, W = q["frames"][0][0].shape
    return srv.add_rig(q["cam0"], q["cam1"], q["R"], q["t"], W, H, q["levels"],
                       lam=q["lam"], huber_eps=q["eps"], **prm)


def _outs(q):
    # pinned host buffers, so that the server's copies are asynchronous and
    # the rigs' work really overlaps on the device
    import torch
    H, W = q["frames"][0][0].shape
    return (torch.empty((H, W), dtype=torch.float32).pin_memory(),
            torch.empty((H, W), dtype=torch.float32).pin_memory())


def _pinned(a):
    import torch
    return torch.from_numpy(a).pin_memory()


def _lone_chain(q, cold_every=False, warm_mode=1, **prm):
    """The same frames through one fs_handle: cold first frame, then warm
    starts from the previous result (fs_solve_continue for warm_mode 1, the
    previous disparity as d_init for 0), or every frame cold."""
    import paper_1909_07545_gb300 as fsb
    H, W = q["frames"][0][0].shape
    s = fsb.Solver(q["cam0"], q["cam1"], q["R"], q["t"], W, H, q["levels"], lam=q["lam"],
                   huber_eps=q["eps"], use_graph=1, **prm)
    res, prev = [], None
    for I0, I1, _ in q["frames"]:
        if prev is None or cold_every:
            d, z = s.solve(I0, I1, *COLD)
        elif warm_mode == 1:
            d, z = s.solve_continue(I0, I1, *WARM)
        else:
            d, z = s.solve(I0, I1, *WARM, init=prev)
        prev = d.clone()
        res.append((np64(d), np64(z)))
    s.close()
    return res


@pytest.mark.parametrize("warm_mode", [1, 0])
def test_served_in_a_mix_equals_served_alone_and_lone_handle(rigs, warm_mode):
    srv = _server(max_inflight=3, warm_mode=warm_mode)
    ids = [_add(srv, q) for q in rigs]
    outs = {}
    reqs = []
    for k in range(3):                          # frame-major: the rigs interleave
        for r, q in zip(ids, rigs):
            d, z = _outs(q)
            I0, I1, _ = q["frames"][k]
            reqs.append(srv.submit(r, _pinned(I0), _pinned(I1), d, z))
            outs[(r, k)] = (d.numpy(), z.numpy())
    lat = [srv.wait(x) for x in reqs]
    st = srv.stats()
    assert st["completed"] == 9 and st["failed"] == 0 and st["cold"] == 3
    assert all(v > 0 for v in lat) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()

    for r, q in zip(ids, rigs):
        alone = _server(max_inflight=1, warm_mode=warm_mode)
        a = _add(alone, q)
        chain = _lone_chain(q, warm_mode=warm_mode)
        for k in range(3):
            d, z = _outs(q)
            I0, I1, _ = q["frames"][k]
            alone.wait(alone.submit(a, I0, I1, d, z))
            d, z = d.numpy(), z.numpy()
            md, mz = outs[(r, k)]
            assert np.array_equal(md, d), (r, k)
            assert np.array_equal(mz, z, equal_nan=True), (r, k)
            assert np.array_equal(md.astype(np.float64), chain[k][0]), (r, k)
            assert np.array_equal(mz.astype(np.float64), chain[k][1], equal_nan=True), (r, k)
        alone.close()


def test_concurrent_waiters_while_submitting(rigs):
    # one waiter thread per rig sits in fs_server_wait while the main thread
    # keeps submitting, so the server's request table grows (and rehashes)
    # under the sleeping waiters; every request completes, with the bits of
    # the same requests waited for one by one from a single thread
    import queue
    import threading
    seq = [0, 1, 2, 1, 0, 1, 2, 1]

    def run(concurrent):
        srv = _server(max_inflight=2)
        ids = [_add(srv, q) for q in rigs]
        outs, reqs, errs = {}, [], []
        qs = [queue.Queue() for _ in rigs]

        def waiter(i):
            while True:
                x = qs[i].get()
                if x is None:
                    return
                try:
                    srv.wait(x)
                except Exception as e:        # reported below
                    errs.append(e)

        ths = [threading.Thread(target=waiter, args=(i,)) for i in range(len(rigs))]
        if concurrent:
            for t in ths:
                t.start()
        for k, f in enumerate(seq):
            for i, (r, q) in enumerate(zip(ids, rigs)):
                d, z = _outs(q)
                I0, I1, _ = q["frames"][f]
                x = srv.submit(r, _pinned(I0), _pinned(I1), d, z)
                outs[(i, k)] = (d, z)
                (qs[i].put if concurrent else reqs.append)(x)
        if concurrent:
            for qq in qs:
                qq.put(None)
            for t in ths:
                t.join()
        else:
            for x in reqs:
                srv.wait(x)
        st = srv.stats()
        srv.close()
        return outs, st, errs

    a, st, errs = run(True)
    assert not errs, errs
    assert st["completed"] == len(seq) * len(rigs) and st["failed"] == 0
    b, _, _ = run(False)
    for key in a:
        assert np.array_equal(a[key][0].numpy(), b[key][0].numpy()), key
        assert np.array_equal(a[key][1].numpy(), b[key][1].numpy(), equal_nan=True), key


def test_served_under_guard_bands(rigs, monkeypatch):
    # FS_GUARD_BANDS=1: every rig handle the server makes has guard bands and
    # every served solve ends with fs_guard_check, whose failure fails the
    # request; results are the same bits as the lone handle's chain
    monkeypatch.setenv("FS_GUARD_BANDS", "1")
    srv = _server(max_inflight=3, warm_mode=1)
    ids = [_add(srv, q) for q in rigs]
    outs, reqs = {}, []
    for k in range(3):
        for r, q in zip(ids, rigs):
            d, z = _outs(q)
            I0, I1, _ = q["frames"][k]
            reqs.append(srv.submit(r, _pinned(I0), _pinned(I1), d, z))
            outs[(r, k)] = (d.numpy(), z.numpy())
    for x in reqs:
        srv.wait(x)
    st = srv.stats()
    assert st["completed"] == 9 and st["failed"] == 0
    srv.close()
    monkeypatch.delenv("FS_GUARD_BANDS")
    for r, q in zip(ids, rigs):
        chain = _lone_chain(q, warm_mode=1)
        for k in range(3):
            assert np.array_equal(outs[(r, k)][0].astype(np.float64), chain[k][0]), (r, k)


def test_budget_admission_evicts_idle_rigs_lru(rigs):
    import paper_1909_07545_gb300 as fsb
    A, B = rigs[0], rigs[2]
    need = []
    for q in (A, B):
        H, W = q["frames"][0][0].shape
        need.append(fsb.state_bytes(W, H, q["levels"]) + 4 * W * H * 4)
    srv = _server(budget_bytes=max(need) + 1, max_inflight=4)   # room for one rig at a time
    a, b = _add(srv, A), _add(srv, B)
    order = [(a, A, 0), (b, B, 0), (a, A, 1), (b, B, 1)]
    res = []
    for r, q, k in order:
        d, z = _outs(q)
        I0, I1, _ = q["frames"][k]
        res.append((srv.submit(r, I0, I1, d, z), d.numpy(), z.numpy()))
    for x, _, _ in res:
        srv.wait(x)
    st = srv.stats()
    # every request had to evict the other rig, so every request was cold
    assert st["cold"] == 4 and st["evictions"] == 3 and st["failed"] == 0
    assert st["peak_resident_bytes"] <= max(need) + 1
    srv.close()
    cold = {id(A): _lone_chain(A, cold_every=True), id(B): _lone_chain(B, cold_every=True)}
    for (r, q, k), (_, d, z) in zip(order, res):
        assert np.array_equal(d.astype(np.float64), cold[id(q)][k][0]), (r, k)
        assert np.array_equal(z.astype(np.float64), cold[id(q)][k][1], equal_nan=True), (r, k)


def test_server_rejects_bad_requests(rigs):
    import paper_1909_07545_gb300 as fsb
    q = rigs[0]
    srv = _server(budget_bytes=1 << 20)        # 1 MiB: no rig fits
    with pytest.raises(fsb.FsError) as e:
        _add(srv, q)
    assert e.value.status == -2
    srv.close()
    srv = _server()
    r = _add(srv, q)
    I0, I1, _ = q["frames"][0]
    assert srv.lib.fs_server_wait(srv.s, 12345, 0.0, None) == -1       # unknown request
    rid = ctypes.c_longlong()
    assert srv.lib.fs_server_submit(srv.s, 7, I0.ctypes.data, I1.ctypes.data, None, None,
                                    ctypes.byref(rid)) == -1               # unknown rig
    bad = dict(q["cam0"], model="kb", k=[0, 0, 0, -0.05], fov_deg=190.0)
    with pytest.raises(fsb.FsError) as e:
        srv.add_rig(bad, q["cam1"], q["R"], q["t"], 128, 128, 2)
    assert e.value.status == -4
    srv.wait(srv.submit(r, I0, I1))
    srv.close()


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_served_16bit_chain_is_as_close_as_the_storage_allows(kind, rigs):
    # a cold frame then a warm-started frame through the server with 16-bit
    # storage, against the FP64 oracle's own chain; the gate is the one of
    # the 16-bit batch path: mean and 99th percentile of |dd| within 3x of
    # the oracle's response to rounding its level images to the same format
    import torch
    dt = {"f16": torch.float16, "bf16": torch.bfloat16}[kind]
    rnd = lambda a: torch.as_tensor(a, dtype=torch.float32).to(dt).to(torch.float64).numpy()
    q = rigs[0]
    srv = _server(max_inflight=2)
    r = _add(srv, q, storage=kind)
    got = []
    for k in range(2):
        d, z = _outs(q)
        I0, I1, _ = q["frames"][k]
        srv.wait(srv.submit(r, I0, I1, d, z))
        got.append(d.numpy().astype(np.float64))
    srv.close()
    pair = dict(cam0=q["cam0"], cam1=q["cam1"], R=q["R"], t=q["t"], levels=q["levels"],
                lam=q["lam"], eps=q["eps"])
    ref, probe = [], []
    for k in range(2):
        I0, I1, _ = q["frames"][k]
        p = dict(pair, I0=I0.astype(np.float64), I1=I1.astype(np.float64))
        w, it = COLD if k == 0 else WARM
        ref.append(oracle_solve(p, warps=w, iters=it,
                                d_init=None if k == 0 else ref[-1]["disp"]))
        probe.append(oracle_solve(p, warps=w, iters=it,
                                  level_hook=lambda l, a, b: (rnd(a), rnd(b)),
                                  d_init=None if k == 0 else probe[-1]["disp"]))
    for k in range(2):
        M = ref[k]["mask"]
        ge = np.abs(got[k] - ref[k]["disp"])[M]
        pe = np.abs(probe[k]["disp"] - ref[k]["disp"])[M]
        rep = dict(kind=kind, frame=k, gpu_mean=float(ge.mean()), probe_mean=float(pe.mean()),
                   gpu_p99=float(np.quantile(ge, 0.99)), probe_p99=float(np.quantile(pe, 0.99)))
        print(rep)
        assert ge.mean() <= 3 * pe.mean(), rep
        assert np.quantile(ge, 0.99) <= 3 * np.quantile(pe, 0.99), rep


def test_cancelled_request_does_not_run(rigs):
    # a queued request can be cancelled; the rig's next request then
    # continues from its last completed frame, as if the cancelled one had
    # never been submitted
    import paper_1909_07545_gb300 as fsb
    q = rigs[0]
    srv = _server(max_inflight=1)
    r = _add(srv, q)
    frames = [q["frames"][k] for k in (0, 1, 2, 0)]
    outs = [_outs(q) for _ in frames]
    ids = [srv.submit(r, _pinned(I0), _pinned(I1), d, z) for (I0, I1, _), (d, z) in
           zip(frames, outs)]
    srv.cancel(ids[2])                         # the rig is still busy with the first two
    with pytest.raises(fsb.FsError):
        srv.cancel(ids[2])                     # no longer queued
    for k, x in enumerate(ids):
        if k == 2:
            with pytest.raises(fsb.FsError) as e:
                srv.wait(x)
            assert e.value.status == -6
        else:
            srv.wait(x)
    st = srv.stats()
    assert st["cancelled"] == 1 and st["completed"] == 3 and st["failed"] == 0
    srv.close()
    # the same frames without the cancelled one, through one handle
    kept = dict(q, frames=[frames[0], frames[1], frames[3]])
    chain = _lone_chain(kept)
    for got, ref in zip([outs[0], outs[1], outs[3]], chain):
        assert np.array_equal(got[0].numpy().astype(np.float64), ref[0])

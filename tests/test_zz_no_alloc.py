"""fs_pd_iterate_noalloc: the primal-dual entry point for callers that cannot
allocate device memory (a real-time thread, a plug-in inside a framework that
owns the device memory pool, a process with a fixed memory cap).

It runs the same iterations as the fs_handle path but keeps its scratch in a
fixed array inside the library.  Checked here, through the C ABI, against
the handle path (fs_buffer_write + fs_run_stage TENSOR/PD) on two calls in a
row with different data and sizes, so a call cannot lean on what the
previous one left in the shared array.  This file runs last (zz) so that a
run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import f32pair, make_solver, np64, ragged_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1909_07545_gb300 import build
    build.build()
    import paper_1909_07545_gb300 as fsb
    return fsb.load_library()


def _inputs(pair, seed):
    rng = np.random.default_rng(seed)
    H, W = pair["I0"].shape
    u = rng.uniform(0, 4, (H, W))
    uw = u + rng.uniform(-0.2, 0.2, (H, W))
    p = rng.uniform(-0.7, 0.7, (2, H, W))
    Iu = rng.uniform(-0.2, 0.2, (H, W))
    rho0 = rng.uniform(-0.05, 0.05, (H, W))
    return u, uw, p, Iu, rho0


def _handle_path(pair, u, uw, p, Iu, rho0, iters, block):
    s = make_solver(pair, block_iters=block)
    M = np64(s.read(0, "MASK")) > 0.5
    u = np.where(M, u, 0.0)
    s.write(0, "I0", pair["I0"])
    s.stage(0, "TENSOR")
    s.write(0, "U", u)
    s.write(0, "UBAR", u)
    s.write(0, "UW", uw)
    s.write(0, "P", p)
    s.write(0, "IU", Iu)
    s.write(0, "RHO0", rho0)
    s.stage(0, "PD", iters)
    out = np64(s.read(0, "U")), np64(s.read(0, "P"))
    s.close()
    return M, u, out


def _noalloc(lib, pair, M, u, uw, p, Iu, rho0, iters, block):
    import torch

    import paper_1909_07545_gb300 as fsb
    H, W = pair["I0"].shape
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")
    tI0, tIu, trho, tuw = dev(pair["I0"]), dev(Iu), dev(rho0), dev(uw)
    tu, tp = dev(u), dev(p)
    tm = torch.as_tensor(M.astype(np.uint8), device="cuda")
    prm = fsb.default_params(lam=pair["lam"], huber_eps=pair["eps"], block_iters=block)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = torch.cuda.current_stream()
    st = lib.fs_pd_iterate_noalloc(ptr(tI0), ptr(tm), ptr(tIu), ptr(trho), ptr(tuw), ptr(tu),
                                   ptr(tp), W, H, iters, ctypes.byref(prm),
                                   ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.fs_last_error().decode()
    stream.synchronize()
    return np64(tu), np64(tp)


def test_noalloc_matches_handle_path_on_two_calls(lib):
    # first call 256 x 256, second a smaller ragged 203 x 157 pair, other data,
    # then a single iteration (one launch: the state is copied back into the
    # caller's buffers).  Both paths run the same kernels on the same inputs,
    # so the results are the same bits.
    cases = [(f32pair(synth.plain_small(0)), 11, 23, 4), (ragged_pair(0), 12, 17, 3),
             (ragged_pair(1), 13, 1, 4)]
    for pair, seed, iters, block in cases:
        u, uw, p, Iu, rho0 = _inputs(pair, seed)
        M, u, (ref_u, ref_p) = _handle_path(pair, u, uw, p, Iu, rho0, iters, block)
        got_u, got_p = _noalloc(lib, pair, M, u, uw, p, Iu, rho0, iters, block)
        assert np.array_equal(got_u, ref_u), iters
        assert np.array_equal(got_p, ref_p), iters


@pytest.mark.parametrize("bad", [dict(regularizer=1), dict(storage=1), dict(storage=2),
                                 dict(accel_gamma=0.1)])
def test_noalloc_rejects_what_it_does_not_compute(lib, bad):
    # TGV, 16-bit storage and the accelerated schedule are fs_handle features:
    # asking for them here is an error, not a silent Huber-TV FP32 run
    import paper_1909_07545_gb300 as fsb
    one = ctypes.c_void_p(16)            # never dereferenced: the checks come first
    prm = fsb.default_params(**bad)
    st = lib.fs_pd_iterate_noalloc(one, one, one, one, one, one, one, 64, 64, 5,
                                   ctypes.byref(prm), None)
    assert st == -1, bad


def test_noalloc_rejects_oversize(lib):
    import paper_1909_07545_gb300 as fsb
    one = ctypes.c_void_p(16)            # never dereferenced: the size check comes first
    st = lib.fs_pd_iterate_noalloc(one, one, one, one, one, one, one, 1024, 1024, 10, None, None)
    assert st == -1
    assert "exceeds the fixed scratch" in lib.fs_last_error().decode()
    assert fsb.default_params() is not None

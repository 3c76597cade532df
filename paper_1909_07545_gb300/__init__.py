"""GB300 non-rectified variational fisheye stereo (Roxas & Oishi) -- Python binding.

Argument marshalling over the C ABI of ``libfs.so`` (``include/fs.h``,
``include/fs_stages.h``, ``include/fs_server.h``); every step of the method
runs in the library's CUDA kernels.  PyTorch only supplies device memory and
the CUDA stream.  The library must have been built
(``paper_1909_07545_gb300.build.build()``); without it, creating a solver
raises instead of falling back to anything.

    Solver   one rig: fs_create / fs_solve / fs_solve_continue / stages
    Batch    many pairs in one CUDA graph (fs_batch_*)
    Server   continuous-batching request server over many rigs (fs_server_*)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Solver", "Batch", "Server", "FsError", "load_library", "default_params",
           "state_bytes", "BUF", "STAGE", "SCHEDULE", "LIB_PATH", "EXPORTED"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfs.so")

MODELS = {"pinhole": 0, "equidistant": 1, "kb": 2, "kannala_brandt": 2, "ucm": 3, "unified": 3,
          "eucm": 4, "enhanced_unified": 4}

BUF = dict(I0=0, I1=1, MASK=2, GAMMA=3, TENSOR=4, STEPS=5, U=6, UBAR=7, UW=8, P=9, W=10,
           IU=11, RHO0=12, G=13, V=14, VBAR=15, Q=16)
BUF_PLANES = {0: 1, 1: 1, 2: 1, 3: 2, 4: 3, 5: 2, 6: 1, 7: 1, 8: 1, 9: 2, 10: 2, 11: 1, 12: 1,
              13: 2, 14: 2, 15: 2, 16: 4}
REGULARIZER = {"huber_tv": 0, "tgv": 1}
DERIV = {"forward": 0, "central": 1}
SCHEDULE = {"auto": 0, "blocking": 1, "persistent": 2}
STAGE = dict(DOWNSAMPLE=0, TENSOR=1, UPSAMPLE=2, WARP=3, PD=4, CLIP=5, TRAJECTORY=6, WARM=7,
             CLIP_WARP=8)

STATUS = {0: "FS_OK", -1: "FS_EINVAL", -2: "FS_ENOMEM", -3: "FS_ECUDA", -4: "FS_ECALIB",
          -5: "FS_ETIMEOUT", -6: "FS_ECANCELLED"}

# every entry point declared in include/*.h
EXPORTED = ["fs_default_params", "fs_create", "fs_set_pose", "fs_level_size",
            "fs_trajectory_field", "fs_solve", "fs_solve_continue", "fs_solve_host", "fs_destroy",
            "fs_last_error",
            "fs_buffer_read", "fs_buffer_write", "fs_run_stage", "fs_stage_prerotate",
            "fs_stage_depth", "fs_timing_enable", "fs_timing_read", "fs_pd_iterate_noalloc",
            "fs_batch_create", "fs_batch_solve", "fs_batch_set_finest_limit",
            "fs_batch_autotune",
            "fs_batch_destroy", "fs_autotune", "fs_set_schedule", "fs_energy", "fs_state_bytes",
            "fs_guard_check", "fs_guard_clobber", "fs_set_wait_limit", "fs_persist_stall",
            "fs_check_waits",
            "fs_server_default_config", "fs_server_create", "fs_server_add_rig",
            "fs_server_submit", "fs_server_wait", "fs_server_cancel", "fs_server_drain",
            "fs_server_stats_read",
            "fs_server_evict_all", "fs_server_destroy"]


class FsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class FsCalib(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("k", ctypes.c_double * 4),
                ("fov_deg", ctypes.c_double)]


class FsPose(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


class FsParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("huber_eps", ctypes.c_float),
                ("du_max", ctypes.c_float), ("beta", ctypes.c_float), ("eta", ctypes.c_float),
                ("theta", ctypes.c_float), ("precond", ctypes.c_int),
                ("block_iters", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("pd_schedule", ctypes.c_int), ("storage", ctypes.c_int),
                ("regularizer", ctypes.c_int), ("alpha0", ctypes.c_float),
                ("alpha1", ctypes.c_float), ("deriv", ctypes.c_int),
                ("accel_gamma", ctypes.c_float)]


_PARAM_FIELDS = {f[0] for f in FsParams._fields_}


class FsServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("warps", ctypes.c_int), ("iters", ctypes.c_int),
                ("cold_warps", ctypes.c_int), ("cold_iters", ctypes.c_int),
                ("warm_mode", ctypes.c_int), ("autotune", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class FsServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("cold", ctypes.c_longlong),
                ("evictions", ctypes.c_longlong), ("cancelled", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("frames_per_s", ctypes.c_double),
                ("resident_bytes", ctypes.c_size_t), ("peak_resident_bytes", ctypes.c_size_t)]


_lib = None
_P = ctypes.c_void_p


def load_library():
    """Load libfs.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "paper_1909_07545_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "fs_default_params": [ctypes.POINTER(FsParams)],
        "fs_create": [ctypes.POINTER(FsCalib), ctypes.POINTER(FsPose), i, i, i,
                      ctypes.POINTER(FsParams), _P, ctypes.POINTER(_P)],
        "fs_set_pose": [_P, ctypes.POINTER(FsPose)],
        "fs_level_size": [_P, i, ctypes.POINTER(i), ctypes.POINTER(i)],
        "fs_trajectory_field": [_P, i, _P],
        "fs_solve": [_P, _P, _P, _P, i, i, _P, _P],
        "fs_solve_continue": [_P, _P, _P, i, i, _P, _P],
        "fs_solve_host": [_P, _P, _P, _P, i, i, _P, _P],
        "fs_destroy": [_P],
        "fs_buffer_read": [_P, i, i, _P],
        "fs_buffer_write": [_P, i, i, _P],
        "fs_run_stage": [_P, i, i, i],
        "fs_stage_prerotate": [_P, _P],
        "fs_stage_depth": [_P, _P, _P],
        "fs_timing_enable": [_P, i],
        "fs_timing_read": [_P, _P, _P, _P, i],
        "fs_pd_iterate_noalloc": [_P, _P, _P, _P, _P, _P, _P, i, i, i,
                                  ctypes.POINTER(FsParams), _P],
        "fs_batch_create": [ctypes.POINTER(_P), i, _P, ctypes.POINTER(_P)],
        "fs_batch_solve": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), i, i,
                           ctypes.POINTER(_P), ctypes.POINTER(_P)],
        "fs_batch_set_finest_limit": [_P, i],
        "fs_batch_autotune": [_P, i, ctypes.POINTER(ctypes.c_int)],
        "fs_batch_destroy": [_P],
        "fs_autotune": [_P, i, _P],
        "fs_set_schedule": [_P, _P],
        "fs_guard_check": [_P],
        "fs_guard_clobber": [_P, i, ctypes.c_size_t, ctypes.POINTER(i)],
        "fs_set_wait_limit": [_P, d],
        "fs_persist_stall": [_P, i],
        "fs_check_waits": [_P],
        "fs_energy": [_P, i, ctypes.POINTER(d)],
        "fs_state_bytes": [i, i, i, ctypes.POINTER(FsParams), ctypes.POINTER(ctypes.c_size_t)],
        "fs_server_default_config": [ctypes.POINTER(FsServerConfig)],
        "fs_server_create": [ctypes.POINTER(FsServerConfig), ctypes.POINTER(_P)],
        "fs_server_add_rig": [_P, ctypes.POINTER(FsCalib), ctypes.POINTER(FsPose), i, i, i,
                              ctypes.POINTER(FsParams), ctypes.POINTER(i)],
        "fs_server_submit": [_P, i, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_longlong)],
        "fs_server_wait": [_P, ctypes.c_longlong, d, ctypes.POINTER(d)],
        "fs_server_drain": [_P, d],
        "fs_server_cancel": [_P, ctypes.c_longlong],
        "fs_server_stats_read": [_P, ctypes.POINTER(FsServerStats), i],
        "fs_server_evict_all": [_P],
        "fs_server_destroy": [_P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fs_last_error.argtypes = []
    lib.fs_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise FsError(status, _lib.fs_last_error().decode())


STORAGE = {"f32": 0, "fp32": 0, "f16": 1, "fp16": 1, "bf16": 2}


def default_params(**overrides) -> FsParams:
    lib = load_library()
    p = FsParams()
    _check(lib.fs_default_params(ctypes.byref(p)))
    for k, v in overrides.items():
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        if k == "regularizer" and isinstance(v, str):
            v = REGULARIZER[v]
        if k == "deriv" and isinstance(v, str):
            v = DERIV[v]
        if k == "pd_schedule" and isinstance(v, str):
            v = SCHEDULE[v]
        name = "lambda_" if k in ("lam", "lambda") else k
        if name not in _PARAM_FIELDS:
            raise TypeError(f"unknown solver parameter {k!r}")
        setattr(p, name, v)
    return p


def _calib(c) -> FsCalib:
    m = c["model"]
    k = list(c.get("k", [0.0] * 4)) + [0.0] * 4
    return FsCalib(MODELS[m] if isinstance(m, str) else int(m), float(c["fx"]), float(c["fy"]),
                   float(c["cx"]), float(c["cy"]), (ctypes.c_double * 4)(*k[:4]),
                   float(c.get("fov_deg", 180.0)))


def _pose(R, t) -> FsPose:
    R = np.asarray(R, dtype=np.float64).reshape(9)
    t = np.asarray(t, dtype=np.float64).reshape(3)
    return FsPose((ctypes.c_double * 9)(*R), (ctypes.c_double * 3)(*t))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Solver:
    """One rig: calibration, pose and per-level device state (fs_create)."""

    def __init__(self, cam0, cam1, R, t, W, H, levels, params=None, stream=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.lib = load_library()
        self.torch = torch
        if params is None:
            params = default_params(**kw)
        self.params = params
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        cams = (FsCalib * 2)(_calib(cam0), _calib(cam1))
        pose = _pose(R, t)
        h = _P()
        _check(self.lib.fs_create(cams, ctypes.byref(pose), int(W), int(H), int(levels),
                                  ctypes.byref(params), _P(stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.W, self.H, self.levels = int(W), int(H), int(levels)

    # ------------------------------------------------------------------ core
    def level_size(self, level):
        w, h = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.fs_level_size(self.h, level, ctypes.byref(w), ctypes.byref(h)))
        return w.value, h.value

    def set_pose(self, R, t):
        _check(self.lib.fs_set_pose(self.h, ctypes.byref(_pose(R, t))))

    def _dev(self, a):
        torch = self.torch
        if isinstance(a, torch.Tensor):
            t = a.to(device="cuda", dtype=torch.float32)
        else:
            t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")
        return t.contiguous()

    def solve(self, I0, I1, warps, iters, init=None, disp=None, depth=None):
        """fs_solve on device tensors (H, W); returns (disparity, depth) tensors."""
        torch = self.torch
        I0 = self._dev(I0)
        I1 = self._dev(I1)
        init = self._dev(init) if init is not None else None
        if disp is None:
            disp = torch.empty((self.H, self.W), device="cuda", dtype=torch.float32)
        if depth is None:
            depth = torch.empty((self.H, self.W), device="cuda", dtype=torch.float32)
        _check(self.lib.fs_solve(self.h, _ptr(I0), _ptr(I1), _ptr(init), int(warps), int(iters),
                                 _ptr(disp), _ptr(depth)))
        self._keep = (I0, I1, init)
        return disp, depth

    def solve_continue(self, I0, I1, warps, iters, disp=None, depth=None):
        """fs_solve_continue: warm start from this handle's own last u and w."""
        torch = self.torch
        I0 = self._dev(I0)
        I1 = self._dev(I1)
        if disp is None:
            disp = torch.empty((self.H, self.W), device="cuda", dtype=torch.float32)
        if depth is None:
            depth = torch.empty((self.H, self.W), device="cuda", dtype=torch.float32)
        _check(self.lib.fs_solve_continue(self.h, _ptr(I0), _ptr(I1), int(warps), int(iters),
                                          _ptr(disp), _ptr(depth)))
        self._keep = (I0, I1)
        return disp, depth

    def solve_host(self, I0, I1, warps, iters, init=None, disp=None, depth=None):
        """fs_solve_host on host float32 arrays (copies inside the call)."""
        def host(a):
            if hasattr(a, "data_ptr"):
                return a
            return np.ascontiguousarray(a, dtype=np.float32)
        I0, I1 = host(I0), host(I1)
        init = host(init) if init is not None else None
        if disp is None:
            disp = np.empty((self.H, self.W), dtype=np.float32)
        if depth is None:
            depth = np.empty((self.H, self.W), dtype=np.float32)

        def p(a):
            if a is None:
                return None
            return _P(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data_as(_P)
        _check(self.lib.fs_solve_host(self.h, p(I0), p(I1), p(init), int(warps), int(iters),
                                      p(disp), p(depth)))
        return disp, depth

    def trajectory_field(self, level=0):
        w, h = self.level_size(level)
        out = self.torch.empty((2, h, w), device="cuda", dtype=self.torch.float32)
        _check(self.lib.fs_trajectory_field(self.h, level, _ptr(out)))
        return out

    # ------------------------------------------------------------------ stages
    def read(self, level, buf):
        b = BUF[buf] if isinstance(buf, str) else int(buf)
        w, h = self.level_size(level)
        out = self.torch.empty((BUF_PLANES[b], h, w), device="cuda", dtype=self.torch.float32)
        _check(self.lib.fs_buffer_read(self.h, level, b, _ptr(out)))
        return out[0] if BUF_PLANES[b] == 1 else out

    def write(self, level, buf, value):
        b = BUF[buf] if isinstance(buf, str) else int(buf)
        w, h = self.level_size(level)
        t = self._dev(value).reshape(BUF_PLANES[b], h, w).contiguous()
        _check(self.lib.fs_buffer_write(self.h, level, b, _ptr(t)))
        self._keep_w = t

    def stage(self, level, stage, count=0):
        s = STAGE[stage] if isinstance(stage, str) else int(stage)
        _check(self.lib.fs_run_stage(self.h, level, s, int(count)))

    def prerotate(self, I1):
        I1 = self._dev(I1)
        _check(self.lib.fs_stage_prerotate(self.h, _ptr(I1)))
        self._keep_p = I1

    def depth(self):
        disp = self.torch.empty((self.H, self.W), device="cuda", dtype=self.torch.float32)
        depth = self.torch.empty_like(disp)
        _check(self.lib.fs_stage_depth(self.h, _ptr(disp), _ptr(depth)))
        return disp, depth

    def autotune(self, iters=20):
        """Pick the primal-dual schedule per level by timing (fs_autotune).
        Returns per level the choice kept, in fs_autotune's encoding
        (include/fs_stages.h): 0 = the whole-level cluster; 8 v + d =
        temporal-blocking depth d (1..8) on footprint v (0..5: 64x64 of 512
        threads, 32x32 of 256, 64x32 of 256, 64x64 of 1024, 32x32 of 1024,
        32x32 of 512), so 1..48; 49..55 = depth 9..15 on 32x32 of 1024
        threads; 56..63 = depth 1..8 on the TMA-staged 64x64 footprints;
        64..71 = depth 1..8 on 64x48 of 768 threads.  TGV handles: 0 = a
        launch per step, 8 v + d = depth d on the five TGV footprints."""
        out = (ctypes.c_int * 8)()
        _check(self.lib.fs_autotune(self.h, int(iters), out))
        return [out[l] for l in range(self.levels)]

    def energy(self, level=0):
        """fs_energy: (total, data, regulariser, L1 residual) of a level's state."""
        out = (ctypes.c_double * 4)()
        _check(self.lib.fs_energy(self.h, int(level), out))
        return tuple(out)

    def set_schedule(self, choice):
        """Set the per-level schedule in autotune()'s encoding (-1 = default)."""
        arr = (ctypes.c_int * 8)(*([int(c) for c in choice] + [-1] * (8 - len(choice))))
        _check(self.lib.fs_set_schedule(self.h, arr))

    def guard_check(self):
        """fs_guard_check: raise FsError if a guard band was overwritten
        (handles created with FS_GUARD_BANDS=1 in the environment)."""
        _check(self.lib.fs_guard_check(self.h))

    def guard_clobber(self, band=-1, offset=0):
        """fs_guard_clobber: zero one byte of a guard band (testing aid);
        returns the number of bands."""
        n = ctypes.c_int()
        _check(self.lib.fs_guard_clobber(self.h, int(band), int(offset), ctypes.byref(n)))
        return n.value

    def set_wait_limit(self, seconds):
        """fs_set_wait_limit: the bound of every wait of the persistent schedule."""
        _check(self.lib.fs_set_wait_limit(self.h, float(seconds)))

    def persist_stall(self, on=True):
        """fs_persist_stall: make a wait of the persistent schedule or of the
        TMA-staged footprints run out (testing aid)."""
        _check(self.lib.fs_persist_stall(self.h, 1 if on else 0))

    def check_waits(self):
        """fs_check_waits: raise FsError (FS_ETIMEOUT) if a copy wait of the
        TMA-staged footprints ran out since the last check."""
        _check(self.lib.fs_check_waits(self.h))

    def timing_enable(self, on=True):
        _check(self.lib.fs_timing_enable(self.h, 1 if on else 0))

    def timing_read(self, reset=False):
        """Per-level primal-dual (ms, launches, pixel-iterations) since the last reset."""
        ms = (ctypes.c_double * 8)()
        n = (ctypes.c_longlong * 8)()
        px = (ctypes.c_double * 8)()
        _check(self.lib.fs_timing_read(self.h, ms, n, px, 1 if reset else 0))
        return [(ms[l], n[l], px[l]) for l in range(self.levels)]

    def close(self):
        if getattr(self, "h", None):
            _check(self.lib.fs_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """fs_batch: one concurrent solve over several Solvers (one pair each)."""

    def __init__(self, solvers, stream=None, finest_limit=0):
        import torch
        self.lib = load_library()
        self.torch = torch
        self.solvers = list(solvers)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        hs = (_P * len(self.solvers))(*[s.h for s in self.solvers])
        b = _P()
        _check(self.lib.fs_batch_create(hs, len(self.solvers), _P(stream.cuda_stream),
                                        ctypes.byref(b)))
        self.b = b
        if finest_limit:
            self.set_finest_limit(finest_limit)

    def set_finest_limit(self, k):
        """At most k pairs on their finest level at once (0: no bound)."""
        _check(self.lib.fs_batch_set_finest_limit(self.b, int(k)))

    def autotune(self, iters=100):
        """fs_batch_autotune: the coarse levels' common schedule for throughput;
        returns the choice kept (-1: the handles' own)."""
        c = ctypes.c_int(-1)
        _check(self.lib.fs_batch_autotune(self.b, int(iters), ctypes.byref(c)))
        return c.value

    def solve(self, I0s, I1s, warps, iters, inits=None, disps=None, depths=None):
        """Device tensors per pair; returns lists of (disparity, depth) tensors."""
        torch = self.torch
        n = len(self.solvers)
        I0s = [s._dev(a) for s, a in zip(self.solvers, I0s)]
        I1s = [s._dev(a) for s, a in zip(self.solvers, I1s)]
        inits = [None] * n if inits is None else \
            [None if a is None else s._dev(a) for s, a in zip(self.solvers, inits)]
        if disps is None:
            disps = [torch.empty((s.H, s.W), device="cuda") for s in self.solvers]
        if depths is None:
            depths = [torch.empty((s.H, s.W), device="cuda") for s in self.solvers]
        arr = lambda ts: (_P * n)(*[None if t is None else t.data_ptr() for t in ts])
        _check(self.lib.fs_batch_solve(self.b, arr(I0s), arr(I1s), arr(inits), int(warps),
                                       int(iters), arr(disps), arr(depths)))
        self._keep = (I0s, I1s, inits)
        return disps, depths

    def close(self):
        if getattr(self, "b", None):
            _check(self.lib.fs_batch_destroy(self.b))
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def state_bytes(W, H, levels, **params) -> int:
    """Device bytes fs_create allocates for a handle (fs_state_bytes); no GPU needed."""
    lib = load_library()
    out = ctypes.c_size_t()
    _check(lib.fs_state_bytes(int(W), int(H), int(levels), ctypes.byref(default_params(**params)),
                              ctypes.byref(out)))
    return out.value


class Server:
    """fs_server: continuous-batching request server over many rigs.

    Each rig keeps its pyramid state and last result resident on the
    device; a rig's first frame is solved cold (cold_warps x cold_iters per
    level), later frames warm-start from its previous result on the finest
    level (warps x iters): warm_mode 1 continues from the finest level's u
    and w, warm_mode 0 restarts from the disparity (w rebuilt along gamma').  Requests of different rigs overlap on the
    GPU; admission is bounded by max_inflight and the device-memory budget.
    Inputs and outputs are host arrays (pinned torch tensors let the copies
    run asynchronously); they are kept referenced until the request is waited
    for.
    """

    def __init__(self, budget_bytes=0, max_inflight=2, warps=3, iters=50, cold_warps=10,
                 cold_iters=100, warm_mode=1, autotune=1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        torch.cuda.init()
        self.lib = load_library()
        self.torch = torch
        cfg = FsServerConfig()
        _check(self.lib.fs_server_default_config(ctypes.byref(cfg)))
        cfg.hbm_budget = int(budget_bytes)
        cfg.max_inflight = int(max_inflight)
        cfg.warps, cfg.iters = int(warps), int(iters)
        cfg.cold_warps, cfg.cold_iters = int(cold_warps), int(cold_iters)
        cfg.warm_mode = int(warm_mode)
        cfg.autotune = int(autotune)
        s = _P()
        _check(self.lib.fs_server_create(ctypes.byref(cfg), ctypes.byref(s)))
        self.s = s
        self.sizes = []
        self._held = {}

    def add_rig(self, cam0, cam1, R, t, W, H, levels, params=None, **kw) -> int:
        if params is None:
            params = default_params(**kw)
        cams = (FsCalib * 2)(_calib(cam0), _calib(cam1))
        rid = ctypes.c_int()
        _check(self.lib.fs_server_add_rig(self.s, cams, ctypes.byref(_pose(R, t)), int(W), int(H),
                                          int(levels), ctypes.byref(params), ctypes.byref(rid)))
        self.sizes.append((int(H), int(W)))
        return rid.value

    def _host(self, a, shape, out=False):
        torch = self.torch
        if isinstance(a, torch.Tensor):
            if a.device.type != "cpu" or a.dtype != torch.float32 or not a.is_contiguous():
                raise ValueError("server buffers must be contiguous float32 CPU tensors")
            t = a
        else:
            if out:
                if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and
                        a.flags["C_CONTIGUOUS"]):
                    raise ValueError("output arrays must be C-contiguous float32")
                t = torch.from_numpy(a)
            else:
                t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
        if tuple(t.shape) != shape:
            raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    def submit(self, rig, I0, I1, disp=None, depth=None) -> int:
        """Queue a pair (host arrays, H x W); returns the request id."""
        shape = self.sizes[rig]
        bufs = [self._host(I0, shape), self._host(I1, shape),
                None if disp is None else self._host(disp, shape, out=True),
                None if depth is None else self._host(depth, shape, out=True)]
        rid = ctypes.c_longlong()
        _check(self.lib.fs_server_submit(self.s, int(rig), *[_ptr(b) for b in bufs],
                                         ctypes.byref(rid)))
        self._held[rid.value] = bufs
        return rid.value

    def wait(self, req, timeout=-1.0) -> float:
        """Block until the request is done; returns its latency in ms."""
        lat = ctypes.c_double()
        st = self.lib.fs_server_wait(self.s, int(req), float(timeout), ctypes.byref(lat))
        if st != -5:                      # FS_ETIMEOUT keeps the request known
            self._held.pop(int(req), None)
        _check(st)
        return lat.value

    def cancel(self, req):
        """Cancel a request that is still queued (FsError if it already ran)."""
        _check(self.lib.fs_server_cancel(self.s, int(req)))

    def drain(self, timeout=-1.0):
        _check(self.lib.fs_server_drain(self.s, float(timeout)))

    def stats(self, reset=False) -> dict:
        st = FsServerStats()
        _check(self.lib.fs_server_stats_read(self.s, ctypes.byref(st), int(bool(reset))))
        return {k: getattr(st, k) for k, _ in FsServerStats._fields_}

    def evict_all(self):
        _check(self.lib.fs_server_evict_all(self.s))

    def close(self):
        if getattr(self, "s", None):
            _check(self.lib.fs_server_destroy(self.s))
            self.s = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""The C ABI: the library builds, loads, exports every declared entry point, and
rejects bad arguments on the host before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1909_07545_gb300 as fsb
from paper_1909_07545_gb300 import build as fsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fs_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    fsbuild.build()
    return fsb.load_library()


def test_every_declared_symbol_is_exported(lib):
    decl = _declared()
    assert "fs_solve" in decl and "fs_create" in decl
    for name in decl:
        assert hasattr(lib, name), name
    assert decl == set(fsb.EXPORTED)


def test_default_params_match_paper(lib):
    p = fsb.default_params()
    assert p.beta == pytest.approx(9.0) and p.eta == pytest.approx(0.85)
    assert p.du_max == pytest.approx(0.2) and p.theta == 1.0 and p.precond == 1
    # and the rest of the defaults fs.h lists for fs_default_params, read from
    # the library itself
    q = fsb.FsParams()
    assert lib.fs_default_params(ctypes.byref(q)) == 0
    assert q.lambda_ == pytest.approx(50.0) and q.huber_eps == pytest.approx(0.01)
    assert (q.block_iters, q.use_graph, q.regularizer, q.deriv, q.storage) == (0, 0, 0, 0, 0)
    assert q.alpha0 == pytest.approx(17.0) and q.alpha1 == pytest.approx(1.2)
    assert q.accel_gamma == 0.0 and q.pd_schedule == 0
    assert lib.fs_default_params(None) == -1


def _create(cams, W=64, H=64, levels=2, prm=None):
    lib = fsb.load_library()
    c = (fsb.FsCalib * 2)(fsb._calib(cams[0]), fsb._calib(cams[1]))
    pose = fsb._pose(np.eye(3), [-0.1, 0, 0])
    h = ctypes.c_void_p()
    st = lib.fs_create(c, ctypes.byref(pose), W, H, levels,
                       ctypes.byref(prm) if prm is not None else None, None, ctypes.byref(h))
    return st, lib.fs_last_error().decode()


EQ = dict(model="equidistant", fx=20.0, fy=20.0, cx=31.5, cy=31.5, fov_deg=180.0)


def test_host_side_validation(lib):
    st, msg = _create([EQ, EQ], levels=0)
    assert st == -1 and "levels" in msg
    st, msg = _create([EQ, EQ], W=64, H=64, levels=6)     # 64 -> 2 px at level 5
    assert st == -1 and "too many levels" in msg
    bad_kb = dict(EQ, model="kb", k=[0, 0, 0, -0.05], fov_deg=190.0)
    st, msg = _create([bad_kb, EQ])
    assert st == -4 and "not increasing" in msg
    pin = dict(EQ, model="pinhole", fov_deg=190.0)
    st, msg = _create([pin, EQ])
    assert st == -4
    neg = dict(EQ, fx=-1.0)
    st, _ = _create([EQ, neg])
    assert st == -4
    # unified: xi >= 0; enhanced unified: 0 <= alpha < 1, beta > 0, and r
    # increasing over the FOV (alpha = 0.95, beta = 1 folds back before 95 deg)
    for bad in (dict(EQ, model="ucm", k=[-0.2, 0, 0, 0]),
                dict(EQ, model="eucm", k=[1.0, 1.0, 0, 0]),
                dict(EQ, model="eucm", k=[0.5, 0.0, 0, 0]),
                dict(EQ, model="eucm", k=[0.95, 1.0, 0, 0], fov_deg=190.0)):
        st, msg = _create([bad, EQ])
        assert st == -4, (bad, msg)
    prm = fsb.default_params(block_iters=9)
    st, msg = _create([EQ, EQ], prm=prm)
    assert st == -1 and "parameter" in msg
    for bad in (dict(regularizer="tgv", storage="f16"), dict(regularizer="tgv", alpha1=0.0),
                dict(regularizer="tgv", alpha0=-1.0), dict(regularizer=2), dict(deriv=2),
                dict(deriv=-1), dict(accel_gamma=-1.0), dict(accel_gamma=0.1),
                dict(accel_gamma=0.1, precond=0, storage="f16"),
                dict(accel_gamma=0.1, precond=0, regularizer="tgv")):
        st, msg = _create([EQ, EQ], prm=fsb.default_params(**bad))
        assert st == -1, bad
    p = fsb.default_params()
    assert p.regularizer == 0 and p.alpha0 == pytest.approx(17.0) and p.alpha1 == pytest.approx(1.2)
    assert p.deriv == 0 and fsb.default_params(deriv="central").deriv == 1   # Eq. 7 by default
    assert p.accel_gamma == 0.0
    with pytest.raises(TypeError):
        fsb.default_params(derivative="central")                   # no silent typo
    h = ctypes.c_void_p()
    assert lib.fs_solve(None, None, None, None, 1, 1, None, None) == -1
    b = ctypes.c_void_p()
    assert lib.fs_batch_create(None, 0, None, ctypes.byref(b)) == -1
    two = (ctypes.c_void_p * 2)(16, 16)
    assert lib.fs_batch_create(two, 2, None, ctypes.byref(b)) == -1     # duplicate handle
    assert "twice" in lib.fs_last_error().decode()
    assert lib.fs_batch_destroy(None) == 0
    assert lib.fs_destroy(None) == 0
    assert lib.fs_create(None, None, 64, 64, 1, None, None, ctypes.byref(h)) == -1


@pytest.mark.parametrize("W,H", [(0, 64), (64, 0), (0, 0), (3, 64), (64, 3), (-8, 64),
                                 (32769, 64), (64, 32769)])
def test_empty_and_out_of_range_sizes_are_rejected_on_the_host(lib, W, H):
    # an empty image, one below the 4-pixel minimum of the coarsest level, or
    # one past the 32768-pixel row limit of the 32-bit plane indexing
    st, msg = _create([EQ, EQ], W=W, H=H, levels=1)
    assert st == -1 and "image size" in msg
    n = ctypes.c_size_t(123)
    assert lib.fs_state_bytes(W, H, 1, None, ctypes.byref(n)) == -1
    assert n.value == 123 and "image size" in lib.fs_last_error().decode()


def test_state_bytes_counts_the_level_planes(lib):
    # mask bytes + 11 FP32 planes + 10 storage-typed planes + 3 float2 planes
    # per level (pitch = width rounded up to 32, planes on 256-byte
    # boundaries), plus the full-resolution calibration field (a float-float
    # pair per pixel: 16 bytes) and the 256-byte status word
    up = lambda v, a: (v + a - 1) // a * a

    def expect(W, H, L, esize):
        total, w, h = 0, W, H
        for l in range(L):
            if l:
                w, h = (w + 1) // 2, (h + 1) // 2
            P = up(w, 32)
            total += up(P * h, 256) + 11 * up(4 * P * h, 256) + 10 * up(esize * P * h, 256) \
                + 6 * up(4 * P * h, 256)
        return total + up(up(W, 32) * H * 16, 256) + 256
    for W, H, L in [(64, 64, 2), (203, 157, 3), (1024, 1024, 5)]:
        assert fsb.state_bytes(W, H, L) == expect(W, H, L, 4)
        assert fsb.state_bytes(W, H, L, storage="f16") == expect(W, H, L, 2)
        assert fsb.state_bytes(W, H, L, storage="bf16") < fsb.state_bytes(W, H, L)
    with pytest.raises(fsb.FsError):
        fsb.state_bytes(64, 64, 6)
    # TGV-L1 adds v, vbar (2 planes each), q (4) and an alternate set of
    # the 12 state planes per level
    extra = sum(20 * up(4 * up((64 + (1 << l) - 1) >> l, 32) * ((64 + (1 << l) - 1) >> l), 256)
                for l in range(2))
    assert fsb.state_bytes(64, 64, 2, regularizer="tgv") == expect(64, 64, 2, 4) + extra


def test_server_config_validation(lib):
    cfg = fsb.FsServerConfig()
    assert lib.fs_server_default_config(ctypes.byref(cfg)) == 0
    assert cfg.hbm_budget == 40 << 30 and cfg.max_inflight == 2
    assert (cfg.warps, cfg.iters, cfg.cold_warps, cfg.cold_iters) == (3, 50, 10, 100)
    assert cfg.warm_mode == 1 and cfg.autotune == 1
    s = ctypes.c_void_p()
    bad = fsb.FsServerConfig(cfg.hbm_budget, 0, 3, 50, 10, 100)
    assert lib.fs_server_create(ctypes.byref(bad), ctypes.byref(s)) == -1
    bad = fsb.FsServerConfig(cfg.hbm_budget, 2, 0, 50, 10, 100)
    assert lib.fs_server_create(ctypes.byref(bad), ctypes.byref(s)) == -1
    bad = fsb.FsServerConfig(cfg.hbm_budget, 2, 3, 50, 10, 100, 2)
    assert lib.fs_server_create(ctypes.byref(bad), ctypes.byref(s)) == -1
    assert "warm_mode" in lib.fs_last_error().decode()
    assert lib.fs_server_create(ctypes.byref(cfg), None) == -1
    assert lib.fs_server_drain(None, 0.0) == -1
    assert lib.fs_server_stats_read(None, None, 0) == -1
    assert lib.fs_server_destroy(None) == 0


def test_headers_are_plain_c99():
    # a C caller's view: the three public headers compile as strict C99
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_check.c")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("bad", [dict(regularizer=1), dict(storage=1), dict(accel_gamma=0.1),
                                 dict(lam=-1.0)])
def test_noalloc_entry_point_rejects_unsupported_options_on_the_host(lib, bad):
    # fs_pd_iterate_noalloc computes Huber-TV iterations on FP32 buffers; the
    # options it does not compute are refused before any device call
    one = ctypes.c_void_p(16)            # never dereferenced
    prm = fsb.default_params(**bad)
    st = lib.fs_pd_iterate_noalloc(one, one, one, one, one, one, one, 64, 64, 5,
                                   ctypes.byref(prm), None)
    assert st == -1, bad
    assert "fs_pd_iterate_noalloc" in lib.fs_last_error().decode()


def test_ctypes_structs_match_the_c_layout(tmp_path):
    # every field the binding declares sits at the offset the C compiler
    # gives it, and each struct has the C size (a field added to a header
    # but not to the binding, or reordered, would shift the rest)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fs_calib": fsb.FsCalib, "fs_pose": fsb.FsPose, "fs_params": fsb.FsParams,
               "fs_server_config": fsb.FsServerConfig, "fs_server_stats": fsb.FsServerStats}
    cname = lambda f: "lambda" if f == "lambda_" else f
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fs.h"',
             '#include "fs_server.h"', 'int main(void) {']
    for s, cls in structs.items():
        lines.append(f'  printf("{s} sizeof %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {cname(f)}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        s, f, v = line.split()
        cls = structs[s]
        want = ctypes.sizeof(cls) if f == "sizeof" else getattr(cls, f).offset
        assert int(v) == want, (s, f, int(v), want)


def _c_signatures():
    """Every fs_* declaration of include/*.h as (name, [parameter kinds]),
    a kind being 'ptr' or the scalar C type."""
    out = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", f)).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\**\s*(fs_\w+)\s*\(([^;{]*?)\)\s*;", src,
                             re.M | re.S):
            params = [p.strip() for p in m.group(2).split(",")]
            if params == ["void"]:
                params = []
            kinds = []
            for p in params:
                if "*" in p or "[" in p:
                    kinds.append("ptr")
                else:
                    kinds.append(" ".join(p.split()[:-1]).replace("const ", ""))
            out[m.group(1)] = kinds
    return out


def test_binding_argtypes_match_the_c_declarations(lib):
    # the arity and every scalar type of each entry point as the binding
    # declares it to ctypes, against the headers
    scalar = {"int": ctypes.c_int, "double": ctypes.c_double, "float": ctypes.c_float,
              "size_t": ctypes.c_size_t, "long long": ctypes.c_longlong}
    sigs = _c_signatures()
    assert set(sigs) == set(fsb.EXPORTED)
    for name, kinds in sigs.items():
        args = getattr(lib, name).argtypes
        assert args is not None and len(args) == len(kinds), (name, kinds, args)
        for k, a in zip(kinds, args):
            if k == "ptr":
                assert a in (ctypes.c_void_p, ctypes.c_char_p) \
                    or issubclass(a, (ctypes._Pointer, ctypes.Array)), (name, k, a)
            else:
                assert a is scalar[k], (name, k, a)


def _c_enum_values():
    """name -> value of every FS_* enumerator and FS_* #define of include/*.h
    (the value given, or one past the previous enumerator)."""
    vals = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", f)).read(), flags=re.S)
        for body in re.findall(r"enum\s*\{([^}]*)\}", src):
            nxt = 0
            for item in [i.strip() for i in body.split(",") if i.strip()]:
                name, _, v = item.partition("=")
                nxt = int(v) if v.strip() else nxt
                vals[name.strip()] = nxt
                nxt += 1
        for name, v in re.findall(r"#define\s+(FS_\w+)\s+(-?\d+)\s*$", src, re.M):
            vals[name] = int(v)
    return vals


def test_binding_constants_match_the_headers():
    c = _c_enum_values()
    for name, v in fsb.BUF.items():
        assert c["FS_BUF_" + name] == v, name
    for name, v in fsb.STAGE.items():
        assert c["FS_STAGE_" + name] == v, name
    for v, name in fsb.STATUS.items():
        assert c[name] == v, name
    assert [c[k] for k in ("FS_PINHOLE", "FS_EQUIDISTANT", "FS_KANNALA_BRANDT", "FS_UNIFIED",
                           "FS_ENHANCED_UNIFIED")] == \
        [fsb.MODELS[k] for k in ("pinhole", "equidistant", "kb", "ucm", "eucm")]
    assert (c["FS_REG_HUBER_TV"], c["FS_REG_TGV"]) == (fsb.REGULARIZER["huber_tv"],
                                                       fsb.REGULARIZER["tgv"])
    assert (c["FS_DERIV_FORWARD"], c["FS_DERIV_CENTRAL"]) == (fsb.DERIV["forward"],
                                                              fsb.DERIV["central"])
    assert c["FS_SCHED_PERSISTENT"] == fsb.SCHEDULE["persistent"]


def test_buffer_plane_counts_match_the_header():
    # fs_stages.h gives each buffer's plane count at the head of its comment
    src = open(os.path.join(ROOT, "include", "fs_stages.h")).read()
    found = re.findall(r"FS_BUF_\w+\s*=\s*(\d+),?\s*/\*\s*(\d+):", src)
    assert len(found) == len(fsb.BUF)
    for v, planes in found:
        assert fsb.BUF_PLANES[int(v)] == int(planes), v


def test_no_cpu_fallback(monkeypatch, tmp_path):
    # without a CUDA device the product classes refuse to run, and without
    # the built library loading it raises: nothing falls back to the CPU
    import torch
    cam = dict(model="equidistant", fx=20.0, fy=20.0, cx=31.5, cy=31.5, fov_deg=180.0)
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError, match="CUDA device"):
        fsb.Solver(cam, cam, np.eye(3), [-0.1, 0, 0], 64, 64, 2)
    with pytest.raises(RuntimeError, match="CUDA device"):
        fsb.Server()
    monkeypatch.setattr(fsb, "_lib", None)
    monkeypatch.setattr(fsb, "LIB_PATH", str(tmp_path / "libfs.so"))
    with pytest.raises(ImportError, match="missing"):
        fsb.load_library()


def test_create_rejects_fuzzed_arguments_without_crashing(lib):
    # seeded random and degenerate calibrations and sizes (NaN, infinities,
    # zero, negative, out-of-range models and fields of view): every call
    # returns an error status and no handle.  The pose always holds a NaN,
    # which fs_create checks after the sizes, levels and calibrations, so
    # every draw runs those checks and none reaches the device.
    import random
    rng = random.Random(11)
    vals = [0.0, -1.0, 1e-300, 1e300, float("nan"), float("inf"), -float("inf"), 1.0, 80.0]
    for _ in range(1500):
        cams = []
        for _ in range(2):
            c = fsb.FsCalib()
            c.model = rng.choice([-1, 0, 1, 2, 3, 4, 5, 99])
            c.fx, c.fy, c.cx, c.cy = (rng.choice(vals) for _ in range(4))
            for i in range(4):
                c.k[i] = rng.choice(vals + [0.03, -0.05])
            c.fov_deg = rng.choice([0.0, -10.0, 179.9, 190.0, 360.0, 720.0, float("nan")])
            cams.append(c)
        pose = fsb._pose(np.eye(3), [-0.1, 0.0, float("nan")])
        h = ctypes.c_void_p()
        st = lib.fs_create((fsb.FsCalib * 2)(*cams), ctypes.byref(pose),
                           rng.choice([0, 3, 64, 100000]), rng.choice([0, 64]),
                           rng.choice([-1, 0, 1, 2, 9]), None, None, ctypes.byref(h))
        assert st in (-1, -4) and not h.value, st

"""GPU kernels against the FP64 oracle, one stage at a time (through the C ABI).

Each test loads the same inputs into the oracle and into a level of an
fs_handle, runs one stage, and compares element by element.  Sizes span
several PD tiles with ragged edges (203 x 157, 256 x 256, 1024 x 1024).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import (f32pair, gpu_level_data, level_calibs, make_solver, np64,
                         oracle_params, ragged_pair, unified_pair)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_07545_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def small():
    return f32pair(synth.plain_small(0))


@pytest.fixture(scope="module")
def ragged():
    return ragged_pair(0)


def _kb_rig(seed=0, W=1024):
    rng = np.random.default_rng(seed)
    k = synth.draw_kb(rng, math.radians(95.0))
    cam = dict(model="kb", fx=320.0 * W / 1024, fy=320.0 * W / 1024, cx=(W - 1) / 2,
               cy=(W - 1) / 2, k=k, fov_deg=190.0)
    from synth.render import rotation
    R = rotation(rng.normal(size=3), math.radians(1.7))
    t = -R @ np.array([0.12, 0.0, 0.0])
    z = np.zeros((W, W))
    return dict(I0=z, I1=z, cam0=cam, cam1=dict(cam), R=R, t=t, levels=5, lam=50.0, eps=0.01)


@pytest.fixture(scope="module")
def unified():
    return {m: unified_pair(5, model0=m, model1="eucm" if m == "ucm" else "ucm")
            for m in ("ucm", "eucm")}


def _ulps(a, b):
    """Distance in float32 units in the last place (same-sign values)."""
    ia = np.float32(a).view(np.int32).astype(np.int64)
    ib = np.float32(b).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


@pytest.mark.parametrize("which", ["small", "ragged", "kb", "ucm", "eucm"])
def test_masks_bit_exact_and_trajectory_field(which, small, ragged, unified):
    pair = {"small": small, "ragged": ragged, "kb": None}.get(which, unified.get(which)) \
        or _kb_rig()
    s = make_solver(pair)
    sizes, cals, masks = level_calibs(pair, pair["levels"])
    tp = oracle.virtual_translation(pair["R"], pair["t"])
    for l in range(pair["levels"]):
        Mg = np64(s.read(l, "MASK")) > 0.5
        assert np.array_equal(Mg, masks[l]), f"mask differs at level {l}"
        g = np64(s.trajectory_field(l)).transpose(1, 2, 0)
        ref = oracle.trajectory_field(cals[l], tp, *sizes[l], masks[l])
        both = (np.linalg.norm(ref, axis=-1) > 0.5) & (np.linalg.norm(g, axis=-1) > 0.5)
        # zero (epipole / off-mask) decisions agree everywhere but at most a
        # pixel or two right at an epipole
        assert np.sum(both != masks[l]) <= 2
        # the GPU computes gamma' in float-float and rounds it once: it is the
        # oracle's field rounded to float32 (a unit vector rounded to float32
        # turns by at most ~6e-8 rad), bit for bit at all but the rare pixels
        # where the two sides straddle a rounding boundary
        ang = np.abs(np.arctan2(g[..., 0] * ref[..., 1] - g[..., 1] * ref[..., 0],
                                np.sum(g * ref, -1)))[both]
        assert ang.max() < 1e-7, (l, ang.max())
        same = np.all(np.float32(g) == np.float32(ref), axis=-1)[both]
        assert same.mean() >= 0.99, (l, same.mean())
    s.close()


@pytest.mark.parametrize("which", ["ragged", "ucm", "eucm"])
def test_prerotation(which, ragged, unified):
    # for "ucm" / "eucm" camera 1 uses the other unified model, so the
    # calibration field also carries the difference of the lenses (Sec. IV-A).
    # The field and the bilinear sample are float-float: the stored image is
    # the oracle's rounded once (within an ulp, mostly bit for bit).
    pair = ragged if which == "ragged" else unified[which]
    s = make_solver(pair)
    s.prerotate(pair["I1"])
    got = np64(s.read(0, "I1"))
    cam0 = oracle.calib_from_dict(pair["cam0"])
    H, W = pair["I0"].shape
    M0 = oracle.fov_mask(cam0, W, H)
    cf = oracle.calibration_field(cam0, oracle.calib_from_dict(pair["cam1"]), pair["R"], W, H, M0)
    ref = oracle.prerotate(pair["I1"], cf)
    assert np.abs(got - ref).max() < 6e-8
    assert (np.float32(got) == np.float32(ref)).mean() >= 0.99
    s.close()


def test_identical_cameras_give_a_zero_calibration_field(small):
    # R = I and camera 1 = camera 0: c(x) = pi_1(R X) - pi_0(X) is exactly 0,
    # so the pre-rotated image is the input, bit for bit
    s = make_solver(small)
    s.prerotate(small["I1"])
    assert np.array_equal(np64(s.read(0, "I1")), small["I1"])
    s.close()


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_downsample(which, small, ragged):
    pair = small if which == "small" else ragged
    s = make_solver(pair)
    sizes, cals, masks = level_calibs(pair, pair["levels"])
    s.write(0, "I0", pair["I0"])
    s.write(0, "I1", pair["I1"])
    r0, r1 = pair["I0"], pair["I1"]
    for l in range(pair["levels"] - 1):
        s.stage(l, "DOWNSAMPLE")
        r0 = oracle.pyramid.downsample_fast(r0, masks[l], *sizes[l + 1])
        r1 = oracle.pyramid.downsample_fast(r1, masks[l], *sizes[l + 1])
        # the levels are carried in float-float: each is the oracle's exact
        # mean rounded once to float32
        for got, ref in ((np64(s.read(l + 1, "I0")), r0), (np64(s.read(l + 1, "I1")), r1)):
            assert _ulps(got, ref).max() <= 1
            assert (np.float32(got) == np.float32(ref)).mean() >= 0.999
    s.close()


@pytest.mark.parametrize("precond", [1, 0])
def test_tensor_and_steps(precond, small, ragged):
    for pair in (small, ragged):
        s = make_solver(pair, precond=precond)
        sizes, cals, masks = level_calibs(pair, pair["levels"])
        prm = oracle_params(pair, precond=bool(precond))
        s.write(0, "I0", pair["I0"])
        s.stage(0, "TENSOR")
        a, b, c = oracle.tensor_sqrt(pair["I0"], masks[0], prm.beta, prm.eta)
        m1, m2 = oracle.grad_masks(masks[0])
        tau, s1, s2 = oracle.precondition(a, b, c, masks[0], m1, m2, prm.precond)
        abc = np64(s.read(0, "TENSOR"))
        M = masks[0]
        for got, ref in zip(abc, (a, b, c)):
            assert np.abs(got - ref)[M].max() < 2e-6
        st = np64(s.read(0, "STEPS"))
        # tau is what holds u outside the mask (0 there): compare inside
        assert np.abs(st[0] - tau)[M].max() < 2e-6 * max(1.0, tau.max())
        assert np.all(st[0][~M] == 0)
        assert np.abs(st[1] - s1).max() < 2e-6 * max(1.0, s1.max())
        s.close()


def _smooth_field(rng, H, W, scale, n=2):
    py, px = np.mgrid[0:H, 0:W].astype(float)
    out = np.zeros((n, H, W))
    for c in range(n):
        for _ in range(3):
            k = rng.normal(size=2) * 0.05
            out[c] += scale * rng.uniform(0.3, 1) * np.sin(k[0] * px + k[1] * py + rng.uniform(0, 6))
    return out


@pytest.mark.parametrize("deriv", ["forward", "central"])
def test_warp_linearize(small, ragged, deriv):
    for pair in (small, ragged):
        s = make_solver(pair, deriv=deriv)
        sizes, cals, masks = level_calibs(pair, pair["levels"])
        rng = np.random.default_rng(7)
        H, W = pair["I0"].shape
        w = _smooth_field(rng, H, W, 3.0)
        u = rng.uniform(0, 5, (H, W))
        s.write(0, "I0", pair["I0"])
        s.write(0, "I1", pair["I1"])
        s.write(0, "W", w)
        s.write(0, "U", u)
        s.stage(0, "WARP")
        gam = np64(s.trajectory_field(0)).transpose(1, 2, 0)
        Iu, rho0, g = oracle.warp_linearize(pair["I0"], pair["I1"], w.transpose(1, 2, 0), gam,
                                            masks[0], deriv)
        assert np.abs(np64(s.read(0, "RHO0")) - rho0).max() < 5e-6
        # where the bicubic sum of unit vectors is short (stencil reaching off
        # the mask or across an epipole) renormalising it amplifies rounding;
        # the comparison is on pixels where |sum| >= 0.2
        py, px = np.mgrid[0:H, 0:W].astype(float)
        graw = oracle.bicubic(gam, px + w[0], py + w[1])
        ok = masks[0] & (np.linalg.norm(graw, axis=-1) >= 0.2)
        assert np.abs(np64(s.read(0, "G")).transpose(1, 2, 0) - g)[ok].max() < 2e-6
        assert np.abs(np64(s.read(0, "IU")) - Iu)[ok].max() < 5e-6
        assert np.array_equal(np64(s.read(0, "UW")), np.float32(u).astype(np.float64))
        assert np.array_equal(np64(s.read(0, "UBAR")), np.float32(u).astype(np.float64))
        s.close()


@pytest.mark.parametrize("prm", [dict(), dict(deriv="central"), dict(storage="f16"),
                                 dict(regularizer="tgv")])
def test_fused_clip_warp_equals_clip_then_warp(small, ragged, prm):
    # what fs_solve runs between two warps (FS_STAGE_CLIP_WARP, one launch)
    # gives the same bits as the clip and warp stages run one after the other
    for pair in (small, ragged):
        outs = []
        for fused in (False, True):
            s = make_solver(pair, **prm)
            s.solve(pair["I0"], pair["I1"], 1, 10)
            if fused:
                s.stage(0, "CLIP_WARP")
            else:
                s.stage(0, "CLIP")
                s.stage(0, "WARP")
            bufs = ["U", "UBAR", "UW", "W", "G", "IU", "RHO0"]
            if prm.get("regularizer") == "tgv":
                bufs += ["V", "VBAR"]
            outs.append([np64(s.read(0, b)) for b in bufs])
            s.close()
        for a, b in zip(*outs):
            assert np.array_equal(a, b)


def _pd_inputs(pair, rng):
    H, W = pair["I0"].shape
    u = rng.uniform(0, 4, (H, W))
    uw = u + rng.uniform(-0.2, 0.2, (H, W))
    p = rng.uniform(-0.7, 0.7, (2, H, W))
    Iu = rng.uniform(-0.2, 0.2, (H, W))
    rho0 = rng.uniform(-0.05, 0.05, (H, W))
    return u, uw, p, Iu, rho0


def _load_pd(s, pair, u, uw, p, Iu, rho0):
    s.write(0, "I0", pair["I0"])
    s.stage(0, "TENSOR")
    M = np64(s.read(0, "MASK")) > 0.5
    u = np.where(M, u, 0.0)
    s.write(0, "U", u)
    s.write(0, "UBAR", u)
    s.write(0, "UW", uw)
    s.write(0, "P", p)
    s.write(0, "IU", Iu)
    s.write(0, "RHO0", rho0)
    return u


@pytest.mark.parametrize("sched,block", [(0, 0), (1, 1), (1, 3), (1, 4), (1, 8)])
def test_pd_iterations_match_oracle(sched, block, small, ragged):
    for pair in (small, ragged):
        rng = np.random.default_rng(11)
        u, uw, p, Iu, rho0 = _pd_inputs(pair, rng)
        s = make_solver(pair, block_iters=block, pd_schedule=sched)
        u = _load_pd(s, pair, u, uw, p, Iu, rho0)
        lv = gpu_level_data(s, 0)
        M = lv["M"]
        f32 = lambda a: np.float32(a).astype(np.float64)
        st = dict(u=f32(u), ubar=f32(u), p1=f32(p[0]), p2=f32(p[1]), Iu=np.where(M, f32(Iu), 0),
                  rho0=np.where(M, f32(rho0), 0), u_w=f32(uw))
        # the GPU stores per-pixel data for every pixel; the oracle's data
        # term is only read inside the mask
        st["Iu"], st["rho0"] = f32(Iu), f32(rho0)
        prm = oracle_params(pair)
        done = 0
        for n in (1, 6, 13):
            s.stage(0, "PD", n)
            for _ in range(n):
                oracle.pd_iteration(st, lv, prm)
            done += n
            gu = np64(s.read(0, "U"))
            gp = np64(s.read(0, "P"))
            tol = 2e-6 * done
            assert np.abs(gu - st["u"]).max() < tol, (block, done)
            assert np.abs(gp[0] - st["p1"]).max() < tol
            assert np.abs(gp[1] - st["p2"]).max() < tol
            assert np.abs(np64(s.read(0, "UBAR")) - st["ubar"]).max() < 2 * tol
        s.close()


@pytest.mark.parametrize("precond", [1, 0])
def test_tgv_iterations_match_oracle(precond, small, ragged):
    # the TGV-L1 primal-dual steps (Eq. 10-11) on loaded state, against the
    # oracle's tgv_iteration with the GPU's own tensor and tau
    for pair in (small, ragged):
        rng = np.random.default_rng(31)
        u, uw, p, Iu, rho0 = _pd_inputs(pair, rng)
        H, W = pair["I0"].shape
        v = rng.uniform(-0.3, 0.3, (2, H, W))
        q = rng.uniform(-2.0, 2.0, (4, H, W))
        s = make_solver(pair, regularizer="tgv", precond=precond)
        u = _load_pd(s, pair, u, uw, p, Iu, rho0)
        lv = gpu_level_data(s, 0)
        M = lv["M"]
        v = np.where(M, v, 0.0)
        q = np.where(M, q, 0.0)
        s.write(0, "V", v)
        s.write(0, "VBAR", v)
        s.write(0, "Q", q)
        f32 = lambda a: np.float32(a).astype(np.float64)
        _, tv, _, sq = oracle.tgv_steps(lv["a"], lv["b"], lv["c"], M, lv["m1"], lv["m2"],
                                        bool(precond))
        sig = np64(s.read(0, "STEPS"))[1]
        if precond:
            lv.update(tau_u=lv["tau"], tau_v=tv, sig_q=sq,
                      sig_p=np.where(M, np.where(sig > 0, sig / (1 + sig), 1.0), 0.0))
        else:
            c = np.where(M, 1.0 / np.sqrt(12.0), 0.0)
            lv.update(tau_u=c, tau_v=c, sig_q=c, sig_p=c)
        st = dict(u=f32(u), ubar=f32(u), p1=f32(p[0]), p2=f32(p[1]), Iu=f32(Iu),
                  rho0=f32(rho0), u_w=f32(uw), v1=f32(v[0]), v2=f32(v[1]), vb1=f32(v[0]),
                  vb2=f32(v[1]), q11=f32(q[0]), q12=f32(q[1]), q21=f32(q[2]), q22=f32(q[3]))
        prm = oracle_params(pair, regularizer="tgv", precond=bool(precond))
        done = 0
        for n in (1, 5, 12):
            s.stage(0, "PD", n)
            for _ in range(n):
                oracle.tgv_iteration(st, lv, prm)
            done += n
            tol = 4e-6 * done
            assert np.abs(np64(s.read(0, "U")) - st["u"]).max() < tol, done
            gp = np64(s.read(0, "P"))
            assert np.abs(gp[0] - st["p1"]).max() < tol and np.abs(gp[1] - st["p2"]).max() < tol
            gv = np64(s.read(0, "V"))
            assert np.abs(gv[0] - st["v1"]).max() < tol and np.abs(gv[1] - st["v2"]).max() < tol
            gq = np64(s.read(0, "Q"))
            for k, name in enumerate(("q11", "q12", "q21", "q22")):
                assert np.abs(gq[k] - st[name]).max() < 4 * tol, name
        s.close()


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_tgv_schedules_are_bit_exact(which, small, ragged):
    # a dual and a primal launch per iteration, and temporal blocking at
    # several depths on each footprint (32 x 32 of 256, 1024, 512 threads;
    # 64 x 32 of 512, 1024), compute the same per-pixel arithmetic
    pair = small if which == "small" else ragged
    H, W = pair["I0"].shape
    outs = []
    for block in (0, 1, 3, 4, 8, 9, 12, 16, 17, 21, 24, 25, 28, 32, 33, 36, 40):
        rng = np.random.default_rng(32)
        u, uw, p, Iu, rho0 = _pd_inputs(pair, rng)
        v = rng.uniform(-0.3, 0.3, (2, H, W))
        q = rng.uniform(-2.0, 2.0, (4, H, W))
        s = make_solver(pair, regularizer="tgv")
        _load_pd(s, pair, u, uw, p, Iu, rho0)
        M = np64(s.read(0, "MASK")) > 0.5
        s.write(0, "V", np.where(M, v, 0.0))
        s.write(0, "VBAR", np.where(M, v, 0.0))
        s.write(0, "Q", np.where(M, q, 0.0))
        s.set_schedule([block] + [-1] * (pair["levels"] - 1))
        s.stage(0, "PD", 17)
        outs.append([np64(s.read(0, b)) for b in ("U", "UBAR", "P", "V", "VBAR", "Q")])
        s.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("reg", ["huber_tv", "tgv"])
def test_energy_reduction_matches_oracle(reg, small, ragged):
    # fs_energy (warp-shuffle reduction on the GPU) against the oracle's
    # energy of the same state, with the GPU's own tensor
    for pair in (small, ragged):
        rng = np.random.default_rng(41)
        u, uw, p, Iu, rho0 = _pd_inputs(pair, rng)
        H, W = pair["I0"].shape
        s = make_solver(pair, regularizer=reg)
        u = _load_pd(s, pair, u, uw, p, Iu, rho0)
        lv = gpu_level_data(s, 0)
        M = lv["M"]
        f32 = lambda a: np.float32(a).astype(np.float64)
        args = (f32(u), f32(uw), f32(Iu), f32(rho0), lv["a"], lv["b"], lv["c"], lv["m1"],
                lv["m2"], M)
        prm = oracle_params(pair, regularizer=reg)
        if reg == "tgv":
            v = np.where(M, rng.uniform(-0.3, 0.3, (2, H, W)), 0.0)
            s.write(0, "V", v)
            ref = oracle.tgv_energy(args[0], f32(v[0]), f32(v[1]), *args[1:], prm.lam,
                                    prm.alpha0, prm.alpha1)
        else:
            ref = oracle.energy(*args, prm.lam, prm.eps)
        total, data, regu, resid = s.energy(0)
        assert abs(total - ref) <= 2e-5 * ref, (reg, total, ref)
        assert abs(data - prm.lam * resid) <= 1e-6 * max(1.0, data)   # per-pixel FP32 products
        s.close()


def test_energy_descends_on_the_gpu(small):
    # the GPU's iterations settle on a lower energy: with scalar steps the
    # energy ends well below its start and stops rising once the iterates
    # settle (Chambolle-Pock is not a descent method step by step)
    rng = np.random.default_rng(42)
    u, uw, p, Iu, rho0 = _pd_inputs(small, rng)
    s = make_solver(small, precond=0)
    _load_pd(s, small, u, uw, p * 0.0, Iu, rho0)
    E = [s.energy(0)[0]]
    for _ in range(60):
        s.stage(0, "PD", 10)
        E.append(s.energy(0)[0])
    E = np.array(E)
    assert E[-1] < 0.8 * E[0]
    assert np.all(np.diff(E[30:]) <= 1e-5 * E[0])
    s.close()


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_pd_schedules_are_bit_exact(which, small, ragged):
    # the whole-level cluster schedule and temporal blocking at every depth
    # compute the same per-pixel arithmetic: results must be identical
    pair = small if which == "small" else ragged
    outs = []
    for sched, block in ((0, 0), (1, 1), (1, 2), (1, 3), (1, 5), (1, 8)):
        rng = np.random.default_rng(12)
        u, uw, p, Iu, rho0 = _pd_inputs(pair, rng)
        s = make_solver(pair, block_iters=block, pd_schedule=sched)
        _load_pd(s, pair, u, uw, p, Iu, rho0)
        s.stage(0, "PD", 17)
        outs.append((np64(s.read(0, "U")), np64(s.read(0, "P")), np64(s.read(0, "UBAR"))))
        s.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_pd_footprints_are_bit_exact(which, small, ragged):
    # every footprint of the tuner's encoding (8 v + depth) on 17 iterations
    # of level 0 from the same state gives the same bits as the default
    # schedule, which the oracle comparison above pins
    pair = small if which == "small" else ragged
    outs = []
    for choice in (-1, 3, 8, 12, 16, 19, 24, 26, 31, 32, 34, 40, 43, 48, 49, 52, 55, 56, 60,
                   62, 63, 64, 67, 70, 71):
        rng = np.random.default_rng(12)
        u, uw, p, Iu, rho0 = _pd_inputs(pair, rng)
        s = make_solver(pair)
        s.set_schedule([choice] + [-1] * (pair["levels"] - 1))
        _load_pd(s, pair, u, uw, p, Iu, rho0)
        s.stage(0, "PD", 17)
        outs.append((np64(s.read(0, "U")), np64(s.read(0, "P")), np64(s.read(0, "UBAR"))))
        s.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_warp_start_constants_equal_the_constant_kernel(storage):
    # The warp-start kernels (k_warp, k_clip_warp) write the iterations'
    # per-pixel constants while they hold I_u, rho0 and u_w; after a buffer
    # write the primal-dual stage recomputes them with k_pd_consts from the
    # stored planes.  Both must give the same bits: the same 9 iterations
    # from the same state, once with each.
    p = f32pair(synth.plain_small(0, W=160, H=128))
    s = make_solver(p, levels=1, storage=storage, pd_schedule=1)
    s.set_schedule([31])
    s.solve(p["I0"], p["I1"], 2, 6)
    s.stage(0, "CLIP_WARP")                      # constants from the fused kernel
    state = {b: np64(s.read(0, b)) for b in ("U", "UBAR", "P")}
    s.stage(0, "PD", 9)
    fused = (np64(s.read(0, "U")), np64(s.read(0, "P")))
    for b, v in state.items():                   # the same state; constants now stale
        s.write(0, b, v)
    s.stage(0, "PD", 9)
    again = (np64(s.read(0, "U")), np64(s.read(0, "P")))
    s.close()
    for a, b in zip(fused, again):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_pd_footprints_agree_across_chained_launches(storage):
    # every footprint at the same depth (5) on 14 iterations of a 64 x 64
    # level: four chained launches of 4, 4, 3 and 3 iterations.  With 16-bit
    # storage the dual is rounded at every launch boundary, so only equal
    # boundaries give equal bits; those must agree whatever the footprint.
    # (Chained launches overlap on an SM when their CTAs are small; state
    # read through L1 then came from a launch two steps back.)
    p = f32pair(synth.plain_small(0, W=64, H=64))
    outs = []
    for choice in (5, 13, 21, 29, 37, 45, 60, 68):   # depth 5 on every footprint
        s = make_solver(p, levels=1, storage=storage, pd_schedule=1)
        s.set_schedule([choice])
        s.solve(p["I0"], p["I1"], 1, 14)
        outs.append((np64(s.read(0, "U")), np64(s.read(0, "P"))))
        s.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_clip_update(ragged):
    pair = ragged
    s = make_solver(pair)
    H, W = pair["I0"].shape
    rng = np.random.default_rng(13)
    M = np64(s.read(0, "MASK")) > 0.5
    u = np.where(M, rng.uniform(0, 3, (H, W)), 0)
    uw = np.where(M, u + rng.uniform(-0.6, 0.6, (H, W)), 0)
    w = rng.uniform(-4, 4, (2, H, W))
    gg = rng.normal(size=(2, H, W))
    gg /= np.linalg.norm(gg, axis=0, keepdims=True)
    s.write(0, "U", u)
    s.write(0, "UW", uw)
    s.write(0, "W", w)
    s.write(0, "G", gg)
    s.stage(0, "CLIP")
    f32 = lambda a: np.float32(a).astype(np.float64)
    un, wn = oracle.clip_update(f32(u), f32(uw), f32(w).transpose(1, 2, 0),
                                f32(gg).transpose(1, 2, 0), 0.2, M)
    assert np.abs(np64(s.read(0, "U"))[M] - un[M]).max() < 1e-6
    assert np.abs(np64(s.read(0, "W")).transpose(1, 2, 0)[M] - wn[M]).max() < 1e-6
    s.close()


def test_upsample(small, ragged):
    for pair in (small, ragged):
        s = make_solver(pair)
        sizes, cals, masks = level_calibs(pair, pair["levels"])
        rng = np.random.default_rng(14)
        Wc, Hc = sizes[1]
        uc = np.where(masks[1], rng.uniform(0, 3, (Hc, Wc)), 0)
        wc = np.where(masks[1], rng.uniform(-2, 2, (2, Hc, Wc)), 0)
        s.write(1, "U", uc)
        s.write(1, "W", wc)
        s.stage(0, "UPSAMPLE")
        f32 = lambda a: np.float32(a).astype(np.float64)
        ru = oracle.upsample(f32(uc), masks[1], *sizes[0], masks[0])
        rw = oracle.upsample(f32(wc).transpose(1, 2, 0), masks[1], *sizes[0], masks[0])
        assert np.abs(np64(s.read(0, "U")) - ru).max() < 2e-6
        assert np.abs(np64(s.read(0, "W")).transpose(1, 2, 0) - rw).max() < 2e-6
        assert np.abs(np64(s.read(0, "P"))).max() == 0.0
        s.close()


@pytest.mark.parametrize("which", ["ragged", "ucm", "eucm"])
def test_depth_triangulation(which, ragged, unified):
    pair = ragged if which == "ragged" else unified[which]
    s = make_solver(pair)
    cam = oracle.calib_from_dict(pair["cam0"])
    H, W = pair["I0"].shape
    M = oracle.fov_mask(cam, W, H)
    tp = oracle.virtual_translation(pair["R"], pair["t"])
    py, px = np.mgrid[0:H, 0:W].astype(float)
    # exact correspondences of points 0.7 - 6 m away
    rng = np.random.default_rng(15)
    rr = rng.uniform(0.7, 6.0, (H, W))
    X = rr[..., None] * oracle.unproject(cam, px, py)
    x1 = oracle.project(cam, X + tp)
    w = np.where(M[..., None], x1 - np.stack([px, py], -1), 0.0)
    u = np.linalg.norm(w, axis=-1)
    s.write(0, "W", w.transpose(2, 0, 1))
    s.write(0, "U", u)
    disp, depth = s.depth()
    disp, depth = np64(disp), np64(depth)
    f32w = np.float32(w).astype(np.float64)
    ref = oracle.triangulate_range(cam, px, py, f32w[..., 0], f32w[..., 1], tp)
    sel = M & (u > 0.5)
    assert np.all(np.isnan(depth[~M])) and np.all(disp[~M] == 0)
    assert np.abs(depth[sel] / ref[sel] - 1).max() < 2e-3
    assert np.median(np.abs(depth[sel] / rr[sel] - 1)) < 1e-3
    s.close()


def test_warm_start_warp_vector(small, ragged):
    # FS_STAGE_WARM: w rebuilt from u by walking the trajectory field
    for pair in (small, ragged):
        rng = np.random.default_rng(21)
        H, W = pair["I0"].shape
        sizes, cals, masks = level_calibs(pair, pair["levels"])
        d = np.float32(np.where(masks[0], 4.0 * rng.uniform(-0.5, 1.0, size=(H, W)), 0.0))
        d = d.astype(np.float64)
        s = make_solver(pair)
        s.write(0, "U", d)
        s.stage(0, "WARM")
        tp = oracle.virtual_translation(pair["R"], pair["t"])
        gamma = np64(s.trajectory_field(0)).transpose(1, 2, 0)
        ref_w = oracle.warm_start_w(d, gamma, masks[0], 0.2)
        got_w = np64(s.read(0, "W")).transpose(1, 2, 0)
        assert np.abs(got_w - ref_w)[masks[0]].max() < 1e-4
        assert np.array_equal(np64(s.read(0, "UW")), d) and np.abs(np64(s.read(0, "P"))).max() == 0
        s.close()

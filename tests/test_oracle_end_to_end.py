"""End-to-end pins for the oracle: paper parameters, renderer/pose convention,
and a rendered fronto-parallel plane recovered at its known depth."""
import json
import os

import numpy as np
import pytest
import scipy.ndimage as nd

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def test_default_parameters_are_the_papers():
    g = json.load(open(GOLDEN))
    prm = oracle.Params()
    assert prm.beta == g["beta"]["value"]
    assert prm.eta == g["eta"]["value"]
    assert prm.du_max == g["du_max_px"]["value"]
    # an 800 x 800 image at scale 2 with minimum width 50 has 5 levels
    sizes = oracle.level_sizes(800, 800, g["pyramid_levels_800"]["value"])
    assert sizes[-1][0] >= g["min_width_px"]["value"]
    assert sizes[-1][0] / g["pyramid_scale"]["value"] < g["min_width_px"]["value"]


def test_renderer_pose_convention_matches_oracle_geometry(small_pair):
    # the ground-truth correspondence pi(P + t') predicted by the oracle's
    # geometry must look at the same scene point in the rendered I1
    p = small_pair
    cam = oracle.calib_from_dict(p["cam0"])
    H, W = p["I0"].shape
    py, px = np.mgrid[0:H, 0:W].astype(float)
    r = oracle.unproject(cam, px, py)
    P = p["gt_range"][..., None] * r
    tp = oracle.virtual_translation(p["R"], p["t"])
    x1 = oracle.project(cam, P + tp)
    M = nd.binary_erosion(oracle.fov_mask(cam, W, H), iterations=6)
    I1s = oracle.bilinear(p["I1"], x1[..., 0], x1[..., 1])
    err = np.abs(I1s - p["I0"])[M]
    wrong = np.abs(oracle.bilinear(p["I1"], px - (x1[..., 0] - px), py)[M] - p["I0"][M])
    assert np.median(err) < 0.01
    assert np.median(wrong) > 3 * np.median(err)


@pytest.mark.parametrize("model", ["equidistant", "pinhole"])
@pytest.mark.parametrize("depth", [1.0, 2.0, 4.0])
def test_fronto_parallel_plane_depth(model, depth):
    p = synth.fronto_plane(0, model=model, depth=depth, cycles_per_px=0.05,
                           baseline=0.2, supersample=4)
    prm = oracle.Params(lam=p["lam"], eps=p["eps"])
    out = oracle.solve(p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"],
                       p["levels"], p["warps"], p["iters"], prm)
    cam = oracle.calib_from_dict(p["cam0"])
    H, W = p["I0"].shape
    py, px = np.mgrid[0:H, 0:W].astype(float)
    r = oracle.unproject(cam, px, py)
    Z = out["depth"] * r[..., 2]
    theta = np.arccos(np.clip(r[..., 2], -1, 1))
    # eroded mask, away from the epipoles at 90 degrees
    sel = nd.binary_erosion(out["mask"], iterations=4) & (theta < np.radians(60))
    rel = Z[sel] / depth - 1.0
    assert abs(np.median(rel)) <= 0.01
    assert np.median(np.abs(rel)) <= 0.025


def test_warm_start_walks_the_trajectory_field():
    # constant field: w = d * gamma exactly; curved field: Euler steps of
    # <= du_max converge to the epipolar curve as the step shrinks
    H, W = 20, 24
    M = np.ones((H, W), bool)
    gam = np.zeros((H, W, 2))
    gam[..., 0] = 0.6
    gam[..., 1] = -0.8
    d = np.linspace(-3, 5, H * W).reshape(H, W)
    w = oracle.warm_start_w(d, gam, M, 0.2)
    assert np.allclose(w[..., 0], 0.6 * d, atol=1e-12)
    assert np.allclose(w[..., 1], -0.8 * d, atol=1e-12)
    cam = oracle.Calib(oracle.camera.EQUIDISTANT, 40.0, 40.0, 63.5, 63.5, fov_deg=180.0)
    Mc = oracle.fov_mask(cam, 128, 128)
    g = oracle.trajectory_field(cam, np.array([-0.1, 0.02, 0.0]), 128, 128, Mc)
    dd = np.where(Mc, 4.0, 0.0)
    coarse = oracle.warm_start_w(dd, g, Mc, 0.2)
    fine = oracle.warm_start_w(dd, g, Mc, 0.02)
    sel = nd.binary_erosion(Mc, iterations=12)
    assert np.abs(coarse - fine)[sel].max() < 0.05
    assert np.abs(np.linalg.norm(fine, axis=-1)[sel] - 4.0).max() < 0.05
    # and the limit is the epipolar curve itself (Sec. III-B): the point 4 px
    # along the projected 3-D line pi(r0 + s t^), s >= 0, traced by brute
    # force (a single straight step d gamma'(x) misses it where the curve bends)
    that = np.array([-0.1, 0.02, 0.0]) / np.hypot(0.1, 0.02)
    ys, xs = np.nonzero(sel)
    rng = np.random.default_rng(7)
    off_straight = 0.0
    for k in rng.choice(len(xs), 24, replace=False):
        x0 = np.array([xs[k], ys[k]], float)
        r0 = oracle.unproject(cam, x0[0], x0[1])
        sv = np.linspace(0.0, 0.5, 20001)
        pts = oracle.project(cam, r0[None, :] + sv[:, None] * that[None, :])
        arc = np.concatenate([[0.0], np.cumsum(np.linalg.norm(np.diff(pts, axis=0), axis=-1))])
        j = int(np.searchsorted(arc, 4.0))
        f = (4.0 - arc[j - 1]) / (arc[j] - arc[j - 1])
        ref = pts[j - 1] + f * (pts[j] - pts[j - 1]) - x0
        assert np.linalg.norm(fine[ys[k], xs[k]] - ref) < 0.02, (xs[k], ys[k])
        off_straight = max(off_straight, float(np.linalg.norm(4.0 * g[ys[k], xs[k]] - ref)))
    assert off_straight > 0.05            # the sample reaches where the curves bend


def test_continuation_with_the_rebuilt_field_is_the_disparity_warm_start():
    # w_init = the field warm_start_w would rebuild from d_init gives the
    # d_init-only warm start exactly; a different w_init changes the result
    p = synth.plain_small(4, W=64, H=64)
    prm = oracle.Params(lam=p["lam"], eps=p["eps"])
    args = (p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"], 2)
    r0 = oracle.solve(*args, 2, 10, prm)
    cam = oracle.calib_from_dict(p["cam0"])
    M = oracle.fov_mask(cam, 64, 64)
    g = oracle.trajectory_field(cam, oracle.virtual_translation(p["R"], p["t"]), 64, 64, M)
    w0 = oracle.warm_start_w(np.where(M, r0["disp"], 0.0), g, M, prm.du_max)
    a = oracle.solve(*args, 1, 8, prm, d_init=r0["disp"])
    b = oracle.solve(*args, 1, 8, prm, d_init=r0["disp"], w_init=w0)
    assert np.array_equal(a["disp"], b["disp"]) and np.array_equal(a["w"], b["w"])
    c = oracle.solve(*args, 1, 8, prm, d_init=r0["disp"], w_init=r0["w"] + 0.5)
    assert np.abs(c["disp"] - a["disp"])[M].max() > 1e-3


def test_image_noise_biases_the_two_derivative_forms_oppositely():
    # reading of Eq. 7 under noise: the forward difference shares I1(x + w)
    # with rho0, so independent image noise pushes every warp's step towards
    # +u and the plane comes out too near; the central difference has no such
    # term, and noise in I_u alone shrinks the steps (the attenuation of a
    # noisy regressor), a smaller bias the other way
    p = synth.fronto_plane(0, model="equidistant", depth=2.0, cycles_per_px=0.05,
                           baseline=0.2, supersample=4)
    rng = np.random.default_rng(5)
    p["I0"] = p["I0"] + rng.normal(0, 0.01, p["I0"].shape)
    p["I1"] = p["I1"] + rng.normal(0, 0.01, p["I1"].shape)
    cam = oracle.calib_from_dict(p["cam0"])
    H, W = p["I0"].shape
    py, px = np.mgrid[0:H, 0:W].astype(float)
    r = oracle.unproject(cam, px, py)
    theta = np.arccos(np.clip(r[..., 2], -1, 1))
    bias = {}
    for deriv in ("forward", "central"):
        prm = oracle.Params(lam=p["lam"], eps=p["eps"], deriv=deriv)
        out = oracle.solve(p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"],
                           p["levels"], p["warps"], p["iters"], prm)
        sel = nd.binary_erosion(out["mask"], iterations=4) & (theta < np.radians(60))
        bias[deriv] = float(np.median(out["depth"][sel] * r[..., 2][sel] / 2.0 - 1.0))
    assert bias["forward"] < -0.05                      # too near: disparity too large
    assert 0.0 < bias["central"] < -bias["forward"]     # too far, by less


def test_accelerated_steps_damp_the_noise_driven_drift():
    # the shrinking tau_k of the accelerated schedule (reading of Sec. IV-C's
    # "theta updated every iteration") takes smaller late steps in each warp,
    # so the forward-difference drift of the noisy plane above is smaller
    p = synth.fronto_plane(0, model="equidistant", depth=2.0, cycles_per_px=0.05,
                           baseline=0.2, supersample=4)
    rng = np.random.default_rng(5)
    p["I0"] = p["I0"] + rng.normal(0, 0.01, p["I0"].shape)
    p["I1"] = p["I1"] + rng.normal(0, 0.01, p["I1"].shape)
    cam = oracle.calib_from_dict(p["cam0"])
    H, W = p["I0"].shape
    py, px = np.mgrid[0:H, 0:W].astype(float)
    r = oracle.unproject(cam, px, py)
    theta = np.arccos(np.clip(r[..., 2], -1, 1))
    bias = []
    for gamma in (0.0, 1.0):
        prm = oracle.Params(lam=p["lam"], eps=p["eps"], precond=False, accel_gamma=gamma)
        out = oracle.solve(p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"],
                           p["levels"], p["warps"], p["iters"], prm)
        sel = nd.binary_erosion(out["mask"], iterations=4) & (theta < np.radians(60))
        bias.append(float(np.median(out["depth"][sel] * r[..., 2][sel] / 2.0 - 1.0)))
    assert bias[0] < bias[1] < 0.0 and bias[1] - bias[0] > 0.01

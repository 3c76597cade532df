"""Pins for the oracle's trajectory field (Sec. III-B, Eq. 6-7), calibration
field (Sec. IV-A) and triangulation (Sec. III-D)."""
import math

import numpy as np
import pytest

from oracle.camera import (Calib, ENHANCED_UNIFIED, EQUIDISTANT, KANNALA_BRANDT, PINHOLE,
                           UNIFIED, project, unproject)
from oracle.geometry import (calibration_field, prerotate, trajectory_field,
                             trajectory_vector, triangulate_range, virtual_translation)
from oracle.pyramid import fov_mask

EQ = Calib(EQUIDISTANT, 80.0, 80.0, 127.5, 127.5, fov_deg=180.0)
KB = Calib(KANNALA_BRANDT, 320.0, 320.0, 511.5, 511.5, (0.03, -0.01, 0.004, 0.001), 190.0)
PH = Calib(PINHOLE, 90.0, 90.0, 63.5, 63.5, fov_deg=100.0)
UCM = Calib(UNIFIED, 150.0, 150.0, 255.5, 255.5, (0.85, 0, 0, 0), 190.0)
EUCM = Calib(ENHANCED_UNIFIED, 160.0, 160.0, 255.5, 255.5, (0.6, 1.15, 0, 0), 190.0)


def _grid(cam, W, H):
    M = fov_mask(cam, W, H)
    return M


def test_pinhole_lateral_translation_gives_constant_field():
    # Sec. III-B: with perspective projection and no rotation the flow
    # direction depends only on t; for t_z = 0 it is (t_x, t_y)/|.| everywhere
    W = H = 128
    M = _grid(PH, W, H)
    t = np.array([0.3, -0.1, 0.0])
    g = trajectory_field(PH, t, W, H, M)
    ref = t[:2] / np.linalg.norm(t[:2])
    assert np.abs(g[M] - ref).max() < 1e-6


def test_pinhole_forward_translation_is_radial_from_epipole():
    W = H = 128
    M = _grid(PH, W, H)
    t = np.array([0.05, 0.02, 0.1])
    g = trajectory_field(PH, t, W, H, M)
    e = np.array([PH.fx * t[0] / t[2] + PH.cx, PH.fy * t[1] / t[2] + PH.cy])
    py, px = np.mgrid[0:H, 0:W].astype(float)
    v = e[None, None, :] - np.stack([px, py], -1)        # towards the epipole
    n = np.linalg.norm(v, axis=-1)
    sel = M & (n > 3.0)
    cross = g[..., 0] * v[..., 1] - g[..., 1] * v[..., 0]
    assert np.abs(cross[sel] / n[sel]).max() < 1e-5      # straight epipolar lines
    dot = np.sum(g * v, -1)
    assert np.all(dot[sel] > 0)                           # t_z > 0: towards e


def test_equidistant_centre_row_points_left():
    # camera-1 centre at +x: t = -C1 = (-b, 0, 0); the centre row is the image
    # of the great circle through the axis and the flow runs along it to -x
    W = H = 256
    M = _grid(EQ, W, H)
    g = trajectory_field(EQ, np.array([-0.1, 0.0, 0.0]), W, H, M)
    row = 127                                             # y = cy - 0.5 (c = 127.5)
    py = np.full(W, 127.5)
    px = np.arange(W, dtype=float)
    gc = trajectory_vector(EQ, np.array([-0.1, 0.0, 0.0]), px, py)
    inside = np.abs(px - EQ.cx) < 80.0 * math.pi / 2 - 2.0
    assert np.abs(gc[inside] - np.array([-1.0, 0.0])).max() < 1e-6
    assert np.all(g[row][M[row]][:, 0] < 0)


@pytest.mark.parametrize("cam,W", [(EQ, 256), (KB, 1024)])
def test_invariance_to_translation_scale_and_depth(cam, W):
    rng = np.random.default_rng(3)
    px = rng.uniform(0.3 * W, 0.7 * W, 200)
    py = rng.uniform(0.3 * W, 0.7 * W, 200)
    t = np.array([0.12, 0.01, -0.02])
    g1 = trajectory_vector(cam, t, px, py)
    g2 = trajectory_vector(cam, 7.0 * t, px, py)
    g3 = trajectory_vector(cam, t, px, py, depth=25.0)
    assert np.abs(g1 - g2).max() < 1e-12
    assert np.abs(g1 - g3).max() < 1e-5


@pytest.mark.parametrize("cam", [EQ, KB, UCM, EUCM])
def test_field_is_tangent_to_traced_epipolar_curves(cam):
    # brute force: project the 3-D points Z r0 + t' for Z from far to near and
    # check that the field at each projected point is tangent to that curve
    t = np.array([-0.12, 0.015, 0.01])
    rng = np.random.default_rng(4)
    W = 2 * cam.cx + 1
    for _ in range(6):
        x0 = rng.uniform(0.35 * W, 0.65 * W, 2)
        r0 = unproject(cam, x0[0], x0[1])
        Z = np.geomspace(50.0, 0.6, 40)
        dZ = 1e-6
        pts = project(cam, Z[:, None] * r0 + t)
        ahead = project(cam, (Z - dZ * Z)[:, None] * r0 + t)
        tan = ahead - pts
        tan /= np.linalg.norm(tan, axis=-1, keepdims=True)
        g = trajectory_vector(cam, t, pts[:, 0], pts[:, 1])
        ang = np.arccos(np.clip(np.sum(tan * g, -1), -1.0, 1.0))
        assert ang.max() < 2e-5


def test_calibration_field_identity_and_axis_roll():
    W = H = 256
    M = fov_mask(EQ, W, H)
    cf = calibration_field(EQ, EQ, np.eye(3), W, H, M)
    assert np.abs(cf).max() < 1e-9
    # a roll by alpha about the optical axis rotates image points about c
    a = math.radians(3.0)
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    cf = calibration_field(EQ, EQ, Rz, W, H, M)
    py, px = np.mgrid[0:H, 0:W].astype(float)
    dx, dy = px - EQ.cx, py - EQ.cy
    ex = math.cos(a) * dx - math.sin(a) * dy - dx
    ey = math.sin(a) * dx + math.cos(a) * dy - dy
    sel = M & (np.hypot(dx, dy) > 1.0)
    assert np.abs(cf[..., 0][sel] - ex[sel]).max() < 1e-8
    assert np.abs(cf[..., 1][sel] - ey[sel]).max() < 1e-8


def test_calibration_field_between_cameras_of_different_focal_length():
    # no rotation, two equidistant cameras with one principal point and focal
    # lengths f and 1.1 f: c(x) = pi_1(X) - pi_0(X) = 0.1 (x - c) exactly
    cam1 = Calib(EQUIDISTANT, 88.0, 88.0, 127.5, 127.5, fov_deg=180.0)
    W = H = 256
    M = fov_mask(EQ, W, H)
    cf = calibration_field(EQ, cam1, np.eye(3), W, H, M)
    py, px = np.mgrid[0:H, 0:W].astype(float)
    assert np.abs(cf[..., 0] - 0.1 * (px - 127.5))[M].max() < 1e-9
    assert np.abs(cf[..., 1] - 0.1 * (py - 127.5))[M].max() < 1e-9


def test_prerotation_of_identity_is_identity():
    rng = np.random.default_rng(5)
    I1 = rng.uniform(0, 1, (40, 50))
    assert np.abs(prerotate(I1, np.zeros((40, 50, 2))) - I1).max() == 0.0


def test_prerotation_samples_the_second_image_at_x_plus_c():
    # I1'(x) = I1(x + c(x)) (Sec. IV-A); bilinear sampling reproduces an
    # affine image exactly, so a constant field (0.25, -0.5) shifts a ramp
    H, W = 12, 16
    py, px = np.mgrid[0:H, 0:W].astype(float)
    I1 = 1.0 + 2.0 * px + 3.0 * py
    cf = np.zeros((H, W, 2))
    cf[..., 0] = 0.25
    cf[..., 1] = -0.5
    out = prerotate(I1, cf)
    ref = 1.0 + 2.0 * (px + 0.25) + 3.0 * (py - 0.5)
    inner = (px + 0.25 <= W - 1) & (py - 0.5 >= 0)
    assert np.abs(out - ref)[inner].max() < 1e-12


@pytest.mark.parametrize("cam", [EQ, KB, PH])
def test_triangulation_recovers_known_points(cam):
    rng = np.random.default_rng(6)
    R = np.eye(3)
    t = np.array([-0.12, 0.02, 0.01])
    tp = virtual_translation(R, t)
    W = 2 * cam.cx + 1
    x0 = rng.uniform(0.4 * W, 0.6 * W, (50, 2))
    rng_true = rng.uniform(0.5, 20.0, 50)
    P = rng_true[:, None] * unproject(cam, x0[:, 0], x0[:, 1])
    x1 = project(cam, P + tp)
    w = x1 - x0
    est = triangulate_range(cam, x0[:, 0], x0[:, 1], w[:, 0], w[:, 1], tp)
    assert np.abs(est / rng_true - 1.0).max() < 1e-8
    zero = triangulate_range(cam, x0[:1, 0], x0[:1, 1], np.zeros(1), np.zeros(1), tp)
    assert np.isinf(zero[0])


def test_virtual_translation_is_rt_t():
    a = math.radians(1.5)
    R = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    # t off the rotation axis: along x alone R t = R^T t, and a transposed R
    # would pass
    t = np.array([-0.12, 0.02, 0.01])
    tp = virtual_translation(R, t)
    assert np.abs(tp - R @ t).max() > 1e-4
    # a point seen by camera 1 (X1 = R X0 + t) is R X1' in the virtual frame
    X0 = np.array([0.3, -0.2, 2.0])
    assert np.allclose(R @ (X0 + tp), R @ X0 + t, atol=1e-15)

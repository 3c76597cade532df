"""Pins for the oracle's sampling (Eq. 9, Sec. III-B) and pyramid (Sec. IV-B)."""
import numpy as np
import pytest

from oracle.camera import Calib, EQUIDISTANT
from oracle.interp import bicubic, bilinear, keys_weight
from oracle.pyramid import (downsample, downsample_fast, fov_mask, level_sizes,
                            scaled_calib, upsample)


def test_bilinear_reproduces_affine_and_samples():
    H, W = 17, 23
    py, px = np.mgrid[0:H, 0:W].astype(float)
    img = 0.3 + 0.02 * px - 0.05 * py
    rng = np.random.default_rng(0)
    x = rng.uniform(0, W - 1, 300)
    y = rng.uniform(0, H - 1, 300)
    assert np.abs(bilinear(img, x, y) - (0.3 + 0.02 * x - 0.05 * y)).max() < 1e-13
    assert np.abs(bilinear(img, px, py) - img).max() == 0.0
    # clamping: outside positions take the value at the clamped position
    assert bilinear(img, np.array([-3.0]), np.array([50.0]))[0] == \
        pytest.approx(img[H - 1, 0], abs=1e-14)


def test_keys_kernel_partition_of_unity_and_quadratic_reproduction():
    s = np.linspace(0, 1, 11)
    tot = sum(keys_weight(s - i) for i in range(-1, 3))
    assert np.abs(tot - 1.0).max() < 1e-14
    H, W = 20, 20
    py, px = np.mgrid[0:H, 0:W].astype(float)
    img = 1.0 + 0.1 * px + 0.2 * py + 0.01 * px * px - 0.02 * px * py + 0.005 * py * py
    rng = np.random.default_rng(1)
    x = rng.uniform(2, W - 3, 200)
    y = rng.uniform(2, H - 3, 200)
    ref = 1.0 + 0.1 * x + 0.2 * y + 0.01 * x * x - 0.02 * x * y + 0.005 * y * y
    assert np.abs(bicubic(img, x, y) - ref).max() < 1e-12
    assert np.abs(bicubic(img, px, py) - img).max() < 1e-13


def test_bicubic_clamps_to_the_edge():
    # a ramp v = x sampled at x = 0.5: the taps at -1, 0, 1, 2 weigh -0.0625,
    # 0.5625, 0.5625, -0.0625 (Keys, a = -0.5), and the tap at -1 reads the
    # edge value v(0) = 0, so the sample is 0.5625 - 0.125 = 0.4375 (0.5 for
    # an unclamped ramp); at the far end, x = 3.5 on 0..4 gives 3.5625
    img = np.tile(np.arange(5.0), (4, 1))
    assert bicubic(img, np.array([0.5]), np.array([1.0]))[0] == pytest.approx(0.4375, abs=1e-15)
    assert bicubic(img, np.array([3.5]), np.array([1.0]))[0] == pytest.approx(3.5625, abs=1e-15)
    assert bicubic(img, np.array([2.5]), np.array([1.0]))[0] == pytest.approx(2.5, abs=1e-15)


def test_level_sizes_and_scaled_calibration():
    assert level_sizes(1024, 1024, 5)[-1] == (64, 64)
    assert level_sizes(1280, 1280, 6)[-1] == (40, 40)
    assert level_sizes(101, 77, 3) == [(101, 77), (51, 39), (26, 20)]
    cam = Calib(EQUIDISTANT, 80.0, 80.0, 127.5, 127.5, fov_deg=180.0)
    c1 = scaled_calib(cam, 1)
    # centre of a 256 image maps to the centre of the 128 image
    assert c1.cx == pytest.approx(63.5) and c1.fx == pytest.approx(40.0)
    # both axes: pixel centres on integers, so c_l = (c + 0.5) 2^-l - 0.5
    # (Sec. IV-B; an off-centre principal point and fx != fy)
    cam2 = Calib(EQUIDISTANT, 80.0, 60.0, 100.0, 140.0, fov_deg=180.0)
    c2 = scaled_calib(cam2, 2)
    assert (c2.fx, c2.fy) == (20.0, 15.0)
    assert (c2.cx, c2.cy) == (24.625, 34.625)


def test_analytic_mask_matches_nearest_neighbour_rescale():
    cam = Calib(EQUIDISTANT, 80.0, 80.0, 127.5, 127.5, fov_deg=180.0)
    M0 = fov_mask(cam, 256, 256)
    M1 = fov_mask(scaled_calib(cam, 1), 128, 128)
    kids = [M0[j::2, i::2] for j in (0, 1) for i in (0, 1)]
    allin = kids[0] & kids[1] & kids[2] & kids[3]
    allout = ~(kids[0] | kids[1] | kids[2] | kids[3])
    assert np.all(M1[allin]) and not np.any(M1[allout])
    assert (allin | allout).mean() > 0.97
    assert 0.7 < M0.mean() < 0.8                # 180 deg circle of radius ~125.7 px


def test_fov_mask_follows_both_focal_lengths():
    # fx = 60, fy = 80: the 180 deg FOV boundary r = pi/2 is an ellipse with
    # semi-axes 94.2 and 125.7 px about (127.5, 127.5); pixel centres half a
    # pixel off the axes, checked just inside and just outside along each
    cam = Calib(EQUIDISTANT, 60.0, 80.0, 127.5, 127.5, fov_deg=180.0)
    M = fov_mask(cam, 256, 256)
    assert M[128, 34] and not M[128, 32]          # dx = -93.5 in, -95.5 out
    assert M[3, 128] and not M[1, 128]            # dy = -124.5 in, -126.5 out


def test_downsample_definition_and_constants():
    rng = np.random.default_rng(2)
    img = rng.uniform(0, 1, (13, 11))
    M = rng.uniform(0, 1, (13, 11)) > 0.3
    a = downsample(img, M, 6, 7)
    b = downsample_fast(img, M, 6, 7)
    assert np.abs(a - b).max() < 1e-15
    assert np.abs(downsample_fast(np.full((13, 11), 0.4), M, 6, 7) - 0.4).max() < 1e-15
    # box mean of a linear ramp equals the ramp at the parent's centre 2X + 0.5
    py, px = np.mgrid[0:16, 0:16].astype(float)
    ramp = 0.1 * px + 0.3 * py
    d = downsample_fast(ramp, np.ones((16, 16), bool), 8, 8)
    Y, X = np.mgrid[0:8, 0:8].astype(float)
    assert np.abs(d - (0.1 * (2 * X + 0.5) + 0.3 * (2 * Y + 0.5))).max() < 1e-13


def test_downsample_averages_only_the_children_inside_the_mask():
    # one parent over the block [[1, 2], [3, 4]]: with the top row in the
    # mask the mean is (1 + 2) / 2, with one child only that child, and with
    # no child in the mask all four count
    img = np.array([[1.0, 2.0], [3.0, 4.0]])
    for f in (downsample, downsample_fast):
        assert f(img, np.array([[True, True], [False, False]]), 1, 1)[0, 0] == 1.5
        assert f(img, np.array([[False, False], [False, True]]), 1, 1)[0, 0] == 4.0
        assert f(img, np.zeros((2, 2), bool), 1, 1)[0, 0] == 2.5


def test_upsample_linear_interior_and_mask():
    Hc = Wc = 10
    Y, X = np.mgrid[0:Hc, 0:Wc].astype(float)
    v = 0.5 + 0.1 * X - 0.2 * Y
    Mc = np.ones((Hc, Wc), bool)
    Mf = np.ones((20, 20), bool)
    Mf[0, 0] = False
    up = upsample(v, Mc, 20, 20, Mf)
    py, px = np.mgrid[0:20, 0:20].astype(float)
    Xc = (px + 0.5) / 2 - 0.5
    Yc = (py + 0.5) / 2 - 0.5
    inner = (Xc >= 0) & (Xc <= Wc - 1) & (Yc >= 0) & (Yc <= Hc - 1) & Mf
    ref = 2.0 * (0.5 + 0.1 * Xc - 0.2 * Yc)
    assert np.abs(up[inner] - ref[inner]).max() < 1e-13
    assert up[0, 0] == 0.0
    # out-of-mask coarse samples get no weight
    Mc2 = Mc.copy()
    Mc2[:, 5:] = False
    v2 = np.where(Mc2, 1.0, 1e6)
    up2 = upsample(v2, Mc2, 20, 20, np.ones((20, 20), bool))
    assert np.abs(up2[:, :10] - 2.0).max() < 1e-12

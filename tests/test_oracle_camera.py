"""Pins for the oracle's camera models (Sec. III-B needs pi; Sec. III-D needs pi^-1)."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle.camera import (Calib, ENHANCED_UNIFIED, EQUIDISTANT, KANNALA_BRANDT, PINHOLE,
                           UNIFIED, is_monotone, project, radial, unproject)

EQ = Calib(EQUIDISTANT, 80.0, 80.0, 127.5, 127.5, fov_deg=180.0)
KB = Calib(KANNALA_BRANDT, 320.0, 318.0, 511.5, 512.5, (0.03, -0.01, 0.004, 0.001), 190.0)
PH = Calib(PINHOLE, 100.0, 110.0, 63.5, 60.0, fov_deg=100.0)
UCM = Calib(UNIFIED, 150.0, 152.0, 127.5, 126.0, (0.85, 0, 0, 0), 190.0)
EUCM = Calib(ENHANCED_UNIFIED, 160.0, 161.0, 127.5, 128.5, (0.6, 1.15, 0, 0), 190.0)


def test_equidistant_closed_form():
    # a ray 45 degrees off-axis in the x-z plane lands f * pi/4 right of centre
    X = np.array([math.sin(math.pi / 4), 0.0, math.cos(math.pi / 4)])
    x = project(EQ, X)
    assert x[0] == pytest.approx(127.5 + 80.0 * math.pi / 4, abs=1e-12)
    assert x[1] == pytest.approx(127.5, abs=1e-12)
    # 90 degrees off-axis straight down: r = f pi/2
    x = project(EQ, np.array([0.0, 1.0, 0.0]))
    assert x[1] == pytest.approx(127.5 + 80.0 * math.pi / 2, abs=1e-12)


def test_pinhole_closed_form():
    X = np.array([0.3, -0.2, 2.0])
    x = project(PH, X)
    assert x[0] == pytest.approx(100.0 * 0.15 + 63.5, abs=1e-12)
    assert x[1] == pytest.approx(110.0 * -0.1 + 60.0, abs=1e-12)


def test_kb_zero_coefficients_is_equidistant():
    kb0 = Calib(KANNALA_BRANDT, 80.0, 80.0, 127.5, 127.5, (0, 0, 0, 0), 180.0)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(100, 3))
    X[:, 2] = np.abs(X[:, 2])
    assert np.allclose(project(kb0, X), project(EQ, X), atol=1e-12)


def test_kb_polynomial_at_one_and_two_radians():
    # at theta = 1 every odd power is 1, so r = 1 + k1 + k2 + k3 + k4; at
    # theta = 2 the powers are 8, 32, 128 and 512 (worked by hand for the
    # coefficients 0.03, -0.01, 0.004, 0.001): a dropped term, a wrong power
    # or two coefficients swapped changes one of the two values
    assert float(radial(KB, 1.0)) == pytest.approx(1.025, abs=1e-14)
    assert float(radial(KB, 2.0)) == pytest.approx(2.944, abs=1e-13)
    # a ray 1 rad off the axis towards +x lands fx r(1) right of the centre
    x = project(KB, np.array([math.sin(1.0), 0.0, math.cos(1.0)]))
    assert x[0] == pytest.approx(511.5 + 320.0 * 1.025, abs=1e-10)
    assert x[1] == pytest.approx(512.5, abs=1e-12)


@pytest.mark.parametrize("cam", [EQ, KB, PH, UCM, EUCM])
def test_round_trip(cam):
    rng = np.random.default_rng(1)
    th = rng.uniform(0.0, cam.theta_max * 0.999, 500)
    ph = rng.uniform(-math.pi, math.pi, 500)
    X = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    x = project(cam, 3.7 * X)
    r = unproject(cam, x[:, 0], x[:, 1])
    assert np.allclose(np.linalg.norm(r, axis=-1), 1.0, atol=1e-14)
    assert np.abs(r - X).max() < 1e-10
    x2 = project(cam, r)
    assert np.abs(x2 - x).max() < 1e-9


def test_kb_inverse_against_brentq():
    rng = np.random.default_rng(2)
    for rn in rng.uniform(0.0, float(radial(KB, KB.theta_max)), 20):
        th = brentq(lambda t: float(radial(KB, t)) - rn, 0.0, KB.theta_max, xtol=1e-15)
        px = KB.cx + KB.fx * rn
        r = unproject(KB, np.array([px]), np.array([KB.cy]))[0]
        assert math.atan2(math.hypot(r[0], r[1]), r[2]) == pytest.approx(th, abs=1e-12)


def test_monotonicity_check():
    assert is_monotone(KB)
    bad = Calib(KANNALA_BRANDT, 320.0, 320.0, 0, 0, (0.0, 0.0, 0.0, -0.05), 190.0)
    assert not is_monotone(bad)


def _rays(n, th_max, seed):
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, th_max, n)
    ph = rng.uniform(-math.pi, math.pi, n)
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)


def test_unified_special_cases():
    # xi = 0 is the pinhole model; xi = 1 is the stereographic model
    # r = tan(theta / 2)
    X = _rays(200, 1.2, 5)
    ucm0 = Calib(UNIFIED, 100.0, 110.0, 63.5, 60.0, (0, 0, 0, 0), 100.0)
    assert np.allclose(project(ucm0, X), project(PH, X), atol=1e-10)
    th = np.linspace(0.0, 1.6, 50)
    st = Calib(UNIFIED, 1.0, 1.0, 0.0, 0.0, (1.0, 0, 0, 0), 190.0)
    assert np.allclose(radial(st, th), np.tan(th / 2.0), atol=1e-14)
    # the model in its usual form m = (X, Y) / (Z + xi |X|), on scaled points
    P = 2.3 * _rays(200, UCM.theta_max, 6)
    m = P[:, :2] / (P[:, 2:] + 0.85 * np.linalg.norm(P, axis=-1, keepdims=True))
    ref = np.stack([150.0 * m[:, 0] + 127.5, 152.0 * m[:, 1] + 126.0], -1)
    assert np.allclose(project(UCM, P), ref, atol=1e-10)


def test_unified_closed_form_unprojection():
    # the literature's closed-form inverse, eta = (xi + sqrt(1 + (1 - xi^2)
    # r^2)) / (1 + r^2), ray ~ (eta m, eta - xi), against the bisection
    rng = np.random.default_rng(7)
    xi = UCM.k[0]
    rmax = float(radial(UCM, UCM.theta_max))
    r = rng.uniform(0.0, rmax * 0.999, 200)
    ph = rng.uniform(-math.pi, math.pi, 200)
    mx, my = r * np.cos(ph), r * np.sin(ph)
    eta = (xi + np.sqrt(1.0 + (1.0 - xi * xi) * r * r)) / (1.0 + r * r)
    ray = np.stack([eta * mx, eta * my, eta - xi], -1)
    ray /= np.linalg.norm(ray, axis=-1, keepdims=True)
    got = unproject(UCM, UCM.cx + UCM.fx * mx, UCM.cy + UCM.fy * my)
    assert np.abs(got - ray).max() < 1e-12


def test_enhanced_unified_special_cases_and_closed_form():
    X = 1.7 * _rays(200, 1.2, 8)
    # alpha = 0 is the pinhole model
    e0 = Calib(ENHANCED_UNIFIED, 100.0, 110.0, 63.5, 60.0, (0.0, 1.3, 0, 0), 100.0)
    assert np.allclose(project(e0, X), project(PH, X), atol=1e-10)
    # beta = 1 is the unified model with xi = alpha / (1 - alpha) and the
    # focal lengths divided by 1 - alpha
    a = 0.6
    e1 = Calib(ENHANCED_UNIFIED, 160.0, 161.0, 127.5, 128.5, (a, 1.0, 0, 0), 190.0)
    u1 = Calib(UNIFIED, 160.0 / (1 - a), 161.0 / (1 - a), 127.5, 128.5, (a / (1 - a), 0, 0, 0),
               190.0)
    Y = 3.1 * _rays(200, e1.theta_max, 9)
    assert np.allclose(project(e1, Y), project(u1, Y), atol=1e-9)
    # usual form m = (X, Y) / (alpha d + (1 - alpha) Z), d = sqrt(beta (X^2 +
    # Y^2) + Z^2), and the closed-form inverse m_z = (1 - beta alpha^2 r^2) /
    # (alpha sqrt(1 - (2 alpha - 1) beta r^2) + 1 - alpha)
    al, be = EUCM.k[0], EUCM.k[1]
    P = 2.0 * _rays(200, EUCM.theta_max, 10)
    d = np.sqrt(be * (P[:, 0] ** 2 + P[:, 1] ** 2) + P[:, 2] ** 2)
    m = P[:, :2] / (al * d + (1 - al) * P[:, 2])[:, None]
    ref = np.stack([EUCM.fx * m[:, 0] + EUCM.cx, EUCM.fy * m[:, 1] + EUCM.cy], -1)
    assert np.allclose(project(EUCM, P), ref, atol=1e-10)
    r2 = np.sum(m * m, -1)
    mz = (1 - be * al * al * r2) / (al * np.sqrt(1 - (2 * al - 1) * be * r2) + 1 - al)
    ray = np.concatenate([m, mz[:, None]], -1)
    ray /= np.linalg.norm(ray, axis=-1, keepdims=True)
    got = unproject(EUCM, ref[:, 0], ref[:, 1])
    assert np.abs(got - ray).max() < 1e-12
    assert np.abs(got - P / 2.0).max() < 1e-12


def test_unified_models_are_monotone_on_their_fov():
    assert is_monotone(UCM) and is_monotone(EUCM)

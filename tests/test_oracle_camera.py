"""Pins for the oracle's camera models (Sec. III-B needs pi; Sec. III-D needs pi^-1)."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle.camera import (Calib, EQUIDISTANT, KANNALA_BRANDT, PINHOLE, is_monotone,
                           project, radial, unproject)

EQ = Calib(EQUIDISTANT, 80.0, 80.0, 127.5, 127.5, fov_deg=180.0)
KB = Calib(KANNALA_BRANDT, 320.0, 318.0, 511.5, 512.5, (0.03, -0.01, 0.004, 0.001), 190.0)
PH = Calib(PINHOLE, 100.0, 110.0, 63.5, 60.0, fov_deg=100.0)


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


@pytest.mark.parametrize("cam", [EQ, KB, PH])
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

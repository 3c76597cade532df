"""Ground-truth disparity of the scene simulator (synth.gt_disparity), pinned
to closed forms: a fronto-parallel plane seen by a pinhole rig translated
along x has the constant disparity f b / Z (straight epipolar lines), and the
optical-axis point of an equidistant rig moves by f atan(b / Z)."""
import math

import numpy as np

import synth


def test_pinhole_plane_disparity_is_f_b_over_z():
    p = synth.fronto_plane(0, model="pinhole", W=64, H=64, depth=2.0, baseline=0.1,
                           supersample=1)
    d, valid = synth.gt_disparity(p, steps=8)
    f = p["cam0"]["fx"]
    assert valid.sum() > 0.9 * valid.size
    assert np.allclose(d[valid], f * 0.1 / 2.0, rtol=1e-9, atol=1e-9)


def test_equidistant_axis_point_moves_by_f_atan_b_over_z():
    p = synth.fronto_plane(1, model="equidistant", W=97, H=97, depth=1.5, baseline=0.1,
                           supersample=1)
    d, valid = synth.gt_disparity(p, steps=256)
    f = p["cam0"]["fx"]
    assert valid[48, 48]
    assert abs(d[48, 48] - f * math.atan(0.1 / 1.5)) < 1e-9
    # off the axis the curve bends: the chord is shorter than the arc
    assert np.all(d[valid] > 0)


def test_error_statistics():
    g = np.array([[1.0, 2.0], [3.0, np.nan]])
    v = np.isfinite(g)
    e = synth.disparity_errors(np.array([[1.5, 4.5], [9.0, 0.0]]), g, v)
    assert e["n"] == 3 and abs(e["epe_mean"] - (0.5 + 2.5 + 6.0) / 3) < 1e-12
    assert e["tau1"] == 2 / 3 and e["tau3"] == 1 / 3 and e["tau5"] == 1 / 3

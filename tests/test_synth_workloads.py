"""The seeded workloads are the configurations they are named for: camera,
rig, pyramid, warps x iterations and weights (rendered here at small sizes;
the generators scale f with the width)."""
import math

import numpy as np
import pytest

import synth
import synth.workloads as wl


def test_plain_small_is_the_256_equidistant_configuration():
    p = synth.plain_small(3, W=64, H=64)
    c = p["cam0"]
    assert c["model"] == "equidistant" and c["fx"] == c["fy"] == 80.0 * 64 / 256
    assert c["fov_deg"] == 180.0 and (c["cx"], c["cy"]) == (31.5, 31.5)
    assert np.array_equal(p["R"], np.eye(3)) and np.allclose(p["t"], [-0.1, 0.0, 0.0])
    assert (p["levels"], p["warps"], p["iters"], p["lam"], p["eps"]) == (3, 5, 50, 50.0, 0.01)
    assert p["I0"].shape == (64, 64) and 0.0 <= p["I0"].min() and p["I0"].max() <= 1.0


def test_plain_kb_is_the_1024_kannala_brandt_configuration():
    p = synth.plain_kb(5, W=64, H=64)
    c = p["cam0"]
    assert c["model"] == "kb" and c["fx"] == 320.0 * 64 / 1024 and c["fov_deg"] == 190.0
    assert max(abs(v) for v in c["k"]) <= 0.05
    assert oracle_monotone(c)
    R = np.asarray(p["R"])
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
    angle = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2))))
    assert angle <= 2.0 + 1e-9
    C1 = -R.T @ np.asarray(p["t"])            # camera-1 centre: 0.12 m along x
    assert np.allclose(C1, [0.12, 0.0, 0.0], atol=1e-12)
    assert (p["levels"], p["warps"], p["iters"], p["lam"], p["eps"]) == (5, 10, 100, 50.0, 0.01)
    assert p["name"] == "plain_kb_64"


def oracle_monotone(cam):
    import oracle
    return oracle.camera.is_monotone(oracle.calib_from_dict(cam))


def test_mixed_2048_is_the_equidistant_generator_at_2048(monkeypatch):
    seen = {}

    def small(seed, W, H, supersample):
        seen.update(seed=seed, W=W, H=H)
        return dict(levels=3, warps=5, iters=50)
    monkeypatch.setattr(wl, "plain_small", small)
    p = wl.mixed_2048(7)
    assert seen == dict(seed=7, W=2048, H=2048)
    assert (p["levels"], p["warps"], p["iters"]) == (6, 10, 100)


@pytest.mark.parametrize("W,L", [(512, 4), (800, 5), (1024, 5), (1280, 6), (640, 5)])
def test_auto_levels_keep_the_coarsest_level_at_least_40_px(W, L):
    assert wl.auto_levels(W) == L
    assert W / 2 ** (L - 1) >= 40 and W / 2 ** L < 40

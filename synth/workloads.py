"""Seeded synthetic workloads: fisheye stereo pairs with known geometry.

The paper's datasets are not available; these scenes stand in for them with
the shapes and value ranges of the evaluated workloads (textured planes and
spheres seen by 180-190 degree fisheye lenses, intensities in [0, 1]).
Every pair is a pure function of (workload, seed, size).

Each pair is a dict:
  I0, I1      float64 (H, W) images in [0, 1], 0 outside the lens FOV
  cam0, cam1  calibration dicts {model, fx, fy, cx, cy, k, fov_deg}
  R, t        pose, X1 = R X0 + t
  gt_range    camera-0 range (m) at pixel centres, NaN outside the FOV
  levels, warps, iters, lam, eps   solver settings of the workload
"""
from __future__ import annotations

import math

import numpy as np

from .render import (kb_is_monotone, make_plane_scene, make_scene, render,
                     rotation)


def _cam(model, W, H, f, fov, k=(0.0, 0.0, 0.0, 0.0)):
    return dict(model=model, fx=float(f), fy=float(f), cx=(W - 1) / 2.0,
                cy=(H - 1) / 2.0, k=[float(v) for v in k], fov_deg=float(fov))


def draw_kb(rng, half_angle, bound=0.05):
    """k1..k4 ~ U(-bound, bound), redrawn until r(theta) is monotone."""
    while True:
        k = rng.uniform(-bound, bound, size=4)
        if kb_is_monotone(k, half_angle):
            return [float(v) for v in k]


def _pair(scene, cam0, cam1, R, C1, W, H, supersample, noise, rng):
    t = -R @ C1
    I0, gt = render(scene, cam0, np.eye(3), np.zeros(3), W, H, supersample, noise, rng)
    I1, _ = render(scene, cam1, R, C1, W, H, supersample, noise, rng)
    return dict(I0=I0, I1=I1, cam0=cam0, cam1=cam1, R=R, t=t, gt_range=gt)


def plain_small(seed=0, W=256, H=256, supersample=2):
    """Equidistant f=80 px 180 deg, 3 planes at 1-5 m, 0.1 m baseline along x."""
    rng = np.random.default_rng(seed)
    f = 80.0 * W / 256.0
    cam = _cam("equidistant", W, H, f, 180.0)
    scene = make_scene(rng, 3, (1.0, 5.0), 5.0, f, kinds=("plane",))
    p = _pair(scene, cam, dict(cam), np.eye(3), np.array([0.1, 0.0, 0.0]), W, H,
              supersample, 0.0, rng)
    p.update(levels=3, warps=5, iters=50, lam=50.0, eps=0.01, name="plain_small_256")
    return p


def plain_kb(seed=0, W=1024, H=1024, supersample=2, levels=5, noise=0.01):
    """Kannala-Brandt f=320 px (at 1024) 190 deg, 20 objects 0.5-20 m, 0.12 m
    baseline + rotation <= 2 deg, Gaussian noise 0.01 (noise=0: the same
    scene and rig without image noise)."""
    rng = np.random.default_rng(seed)
    f = 320.0 * W / 1024.0
    half = math.radians(190.0) / 2.0
    k = draw_kb(rng, half)
    cam = _cam("kb", W, H, f, 190.0, k)
    axis = rng.normal(size=3)
    R = rotation(axis, math.radians(rng.uniform(0.0, 2.0)))
    scene = make_scene(rng, 20, (0.5, 20.0), 20.0, f, kinds=("plane", "sphere"))
    p = _pair(scene, cam, dict(cam), R, np.array([0.12, 0.0, 0.0]), W, H,
              supersample, noise, rng)
    p.update(levels=levels, warps=10, iters=100, lam=50.0, eps=0.01,
             name=f"plain_kb_{W}" if noise == 0.01 else f"plain_kb_{W}_noise{noise:g}")
    return p


def mixed_2048(seed=0, supersample=2):
    """The 180-degree equidistant generator at 2048 x 2048, 6 levels."""
    p = plain_small(seed, 2048, 2048, supersample)
    p.update(levels=6, warps=10, iters=100, name="equidistant_2048")
    return p


def auto_levels(W, min_width=40):
    L = 1
    while W / 2 ** L >= min_width:
        L += 1
    return L


def fronto_plane(seed=0, model="equidistant", W=192, H=192, f=None, depth=2.0,
                 baseline=0.1, supersample=2, cycles_per_px=0.25):
    """A single textured plane Z = depth seen with a pure x translation."""
    rng = np.random.default_rng(seed)
    if model == "pinhole":
        f = f or W / 2.0
        cam = _cam("pinhole", W, H, f, 100.0)
    else:
        f = f or 60.0 * W / 192.0
        cam = _cam("equidistant", W, H, f, 180.0)
    scene = make_plane_scene(rng, depth, f, cycles_per_px=cycles_per_px)
    p = _pair(scene, cam, dict(cam), np.eye(3), np.array([baseline, 0.0, 0.0]), W, H,
              supersample, 0.0, rng)
    p.update(levels=4, warps=8, iters=60, lam=50.0, eps=0.01, name=f"plane_{model}")
    return p


def _smooth_path(rng, n_axes, max_rate, fmin=0.05, fmax=0.3):
    """A function of time: per axis a sum of 3 sinusoids of low frequency,
    amplitudes scaled so that the rate of change (the norm over the axes)
    never exceeds max_rate."""
    f = rng.uniform(fmin, fmax, size=(n_axes, 3))
    ph = rng.uniform(0.0, 2 * math.pi, size=(n_axes, 3))
    # |d/dt sum a_j sin(2 pi f_j t + ph_j)| <= sum a_j 2 pi f_j  (per axis)
    a = max_rate / (3 * 2 * math.pi * f * math.sqrt(n_axes))

    def at(t):
        return (a * np.sin(2 * math.pi * f * t + ph)).sum(axis=1)
    return at


def rig_sequence(seed=0, W=640, H=640, n_frames=3, rate_hz=37.5, supersample=1, noise=0.01,
                 levels=None, n_objects=20):
    """A moving stereo rig: one seeded Kannala-Brandt calibration (f = 320 px
    at 1024, 190 deg), a fixed relative pose (0.12 m baseline along x plus a
    rotation <= 2 deg) and a fixed scene of planes and spheres at 0.5-20 m.
    The rig's camera 0 follows a smooth path (position and rotation vector
    each a sum of 3 low-frequency sinusoids per axis; speed <= 0.5 m/s,
    rotation-vector rate <= 5 deg/s); frame k is rendered at time k / rate_hz.

    Returns dict(cam0, cam1, R, t, levels, frames=[(I0, I1, gt_range), ...]).
    R, t (X1 = R X0 + t) are the rig's, identical for every frame."""
    rng = np.random.default_rng(seed)
    f = 320.0 * W / 1024.0
    half = math.radians(190.0) / 2.0
    cam = _cam("kb", W, H, f, 190.0, draw_kb(rng, half))
    R = rotation(rng.normal(size=3), math.radians(rng.uniform(0.0, 2.0)))
    C1 = np.array([0.12, 0.0, 0.0])
    scene = make_scene(rng, n_objects, (0.5, 20.0), 20.0, f, kinds=("plane", "sphere"))
    pos = _smooth_path(rng, 3, 0.5)
    rot = _smooth_path(rng, 3, math.radians(5.0))
    frames = []
    for k in range(n_frames):
        tk = k / rate_hz
        o = pos(tk)
        rv = rot(tk)
        ang = float(np.linalg.norm(rv))
        R0 = rotation(rv, ang) if ang > 0 else np.eye(3)      # world -> camera 0
        I0, gt = render(scene, cam, R0, o, W, H, supersample, noise, rng)
        # camera 1: X1 = R X0 + t, so world -> camera 1 is R R0 and its
        # centre is o + R0^T C1
        I1, _ = render(scene, cam, R @ R0, o + R0.T @ C1, W, H, supersample, noise, rng)
        frames.append((I0, I1, gt))
    return dict(cam0=cam, cam1=dict(cam), R=R, t=-R @ C1, frames=frames,
                levels=levels or auto_levels(W), lam=50.0, eps=0.01,
                name=f"rig_kb_{W}")


def _project(cam, X):
    """Pixel position of camera-frame points X (..., 3) through the lens."""
    from .render import lens_radius
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    th = np.arctan2(np.hypot(x, y), z)
    phi = np.arctan2(y, x)
    r = lens_radius(cam, th)
    return np.stack([cam["fx"] * r * np.cos(phi) + cam["cx"],
                     cam["fy"] * r * np.sin(phi) + cam["cy"]], -1)


def gt_disparity(pair, steps=64):
    """Ground-truth disparity of a rendered pair: the arc length, in pixels,
    of the path a camera-0 pixel's true 3-D point X traces in the image of a
    camera with camera 0's orientation and lens as that camera's centre moves
    from camera 0's to camera 1's (the point X - s C1, s from 0 to 1; C1 the
    camera-1 centre in camera-0 coordinates).  This is the distance along the
    epipolar curve to the true correspondence after the orientation of camera
    1 is undone.  Polyline of `steps` segments.  Returns (d_gt, valid): valid
    where the pixel sees a finite point inside the lens FOV that stays in
    front of the moving camera and inside its FOV."""
    from .render import lens_rays
    cam = pair["cam0"]
    H, W = pair["I0"].shape
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    rays, valid = lens_rays(cam, px, py)
    rng = pair["gt_range"]
    valid = valid & np.isfinite(rng)
    X = rays * np.where(valid, rng, 1.0)[..., None]
    R = np.asarray(pair["R"], dtype=np.float64)
    C1 = -R.T @ np.asarray(pair["t"], dtype=np.float64)
    half = math.radians(cam["fov_deg"]) / 2.0
    prev = _project(cam, X)
    arc = np.zeros((H, W))
    for k in range(1, steps + 1):
        P = X - (k / steps) * C1
        th = np.arctan2(np.hypot(P[..., 0], P[..., 1]), P[..., 2])
        valid &= th <= half
        cur = _project(cam, P)
        arc += np.linalg.norm(cur - prev, axis=-1)
        prev = cur
    return np.where(valid, arc, np.nan), valid


def disparity_errors(d, d_gt, valid):
    """End-point error statistics against ground truth over `valid`: mean,
    median, and the fractions of erroneous pixels above 1, 3 and 5 px (the
    error measure of the paper's Sec. V, tau > 1 and tau > 5 px)."""
    e = np.abs(np.asarray(d, dtype=np.float64) - d_gt)[valid]
    return dict(epe_mean=float(e.mean()), epe_median=float(np.median(e)),
                tau1=float((e > 1.0).mean()), tau3=float((e > 3.0).mean()),
                tau5=float((e > 5.0).mean()), n=int(valid.sum()))

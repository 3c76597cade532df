"""Camera projection pi and unprojection pi^-1 in float64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

The method only needs *some* projection function pi (Sec. III-B: any model
works as long as pi is defined; the unified, enhanced unified and
Kannala-Brandt models are cited there) and its inverse for triangulation
(Sec. III-D, last paragraph).  Five radially symmetric models are written
out, with s = sin(theta), c = cos(theta):

  pinhole           r(theta) = tan(theta)
  equidistant       r(theta) = theta
  Kannala-Brandt    r(theta) = theta + k1 theta^3 + k2 theta^5 + k3 theta^7 + k4 theta^9
  unified           r(theta) = s / (c + xi)                      (xi = k[0])
  enhanced unified  r(theta) = s / (alpha sqrt(beta s^2 + c^2) + (1 - alpha) c)
                                                     (alpha = k[0], beta = k[1])

with pixel = (fx * r * X/rho + cx, fy * r * Y/rho + cy), rho = |(X, Y)|,
theta = atan2(rho, Z).  Pixel centres sit on integer coordinates.
The unprojection solves r(theta) = |m| by plain bisection on the interval
where r is monotone (the FOV half-angle), which is slow but needs no
argument beyond monotonicity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

PINHOLE, EQUIDISTANT, KANNALA_BRANDT, UNIFIED, ENHANCED_UNIFIED = 0, 1, 2, 3, 4
_MODEL_NAMES = {"pinhole": PINHOLE, "equidistant": EQUIDISTANT,
                "kb": KANNALA_BRANDT, "kannala_brandt": KANNALA_BRANDT,
                "ucm": UNIFIED, "unified": UNIFIED,
                "eucm": ENHANCED_UNIFIED, "enhanced_unified": ENHANCED_UNIFIED}


@dataclass(frozen=True)
class Calib:
    model: int
    fx: float
    fy: float
    cx: float
    cy: float
    k: tuple = (0.0, 0.0, 0.0, 0.0)
    fov_deg: float = 180.0

    @property
    def theta_max(self) -> float:
        return math.radians(self.fov_deg) / 2.0


def calib_from_dict(d) -> Calib:
    """Build a Calib from the plain-dict interchange format of the generators
    (the camera models Sec. III-B admits)."""
    if isinstance(d, Calib):
        return d
    m = d["model"]
    model = _MODEL_NAMES[m] if isinstance(m, str) else int(m)
    k = tuple(float(v) for v in d.get("k", (0.0, 0.0, 0.0, 0.0)))
    k = k + (0.0,) * (4 - len(k))
    return Calib(model, float(d["fx"]), float(d["fy"]), float(d["cx"]),
                 float(d["cy"]), k, float(d.get("fov_deg", 180.0)))


def radial(calib: Calib, theta):
    """Normalised image radius r(theta) of the model: the radial part of the
    projection pi that Sec. III-B needs (any model with a defined pi)."""
    theta = np.asarray(theta, dtype=np.float64)
    if calib.model == PINHOLE:
        return np.tan(theta)
    if calib.model == EQUIDISTANT:
        return theta
    if calib.model == UNIFIED:
        return np.sin(theta) / (np.cos(theta) + calib.k[0])
    if calib.model == ENHANCED_UNIFIED:
        alpha, beta = calib.k[0], calib.k[1]
        s, c = np.sin(theta), np.cos(theta)
        return s / (alpha * np.sqrt(beta * s * s + c * c) + (1.0 - alpha) * c)
    k1, k2, k3, k4 = calib.k
    t2 = theta * theta
    return theta * (1.0 + t2 * (k1 + t2 * (k2 + t2 * (k3 + t2 * k4))))


def fov_radius(calib: Calib) -> float:
    """Normalised radius of the FOV circle, r(theta_max) (the image region
    the method works on, Sec. IV-B's mask)."""
    return float(radial(calib, calib.theta_max))


def project(calib: Calib, X):
    """pi: 3-D points (..., 3) in the camera frame -> pixels (..., 2)
    (Sec. III-A, III-B)."""
    X = np.asarray(X, dtype=np.float64)
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    rho = np.hypot(x, y)
    theta = np.arctan2(rho, z)
    r = radial(calib, theta)
    safe = np.where(rho > 0.0, rho, 1.0)
    mx = np.where(rho > 0.0, r * x / safe, 0.0)
    my = np.where(rho > 0.0, r * y / safe, 0.0)
    return np.stack([calib.fx * mx + calib.cx, calib.fy * my + calib.cy], axis=-1)


def _theta_of_radius(calib: Calib, rn):
    """Solve r(theta) = rn for theta in [0, theta_max] by bisection (FP64): the
    inverse radial map behind pi^-1 (Sec. III-D).

    rn beyond r(theta_max) returns theta_max (callers mask such pixels out).
    """
    rn = np.asarray(rn, dtype=np.float64)
    if calib.model == EQUIDISTANT:
        return rn.copy()
    if calib.model == PINHOLE:
        return np.arctan(rn)
    lo = np.zeros_like(rn)
    hi = np.full_like(rn, calib.theta_max)
    for _ in range(64):
        mid = 0.5 * (lo + hi)
        below = radial(calib, mid) < rn
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def unproject(calib: Calib, px, py):
    """pi^-1: pixel coordinates -> unit rays (..., 3) in the camera frame
    (Sec. III-B, III-D)."""
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    mx = (px - calib.cx) / calib.fx
    my = (py - calib.cy) / calib.fy
    rn = np.hypot(mx, my)
    theta = _theta_of_radius(calib, rn)
    s = np.sin(theta)
    safe = np.where(rn > 0.0, rn, 1.0)
    return np.stack([np.where(rn > 0.0, s * mx / safe, 0.0),
                     np.where(rn > 0.0, s * my / safe, 0.0),
                     np.cos(theta)], axis=-1)


def is_monotone(calib: Calib, samples: int = 10000) -> bool:
    """True when r(theta) strictly increases on [0, theta_max] (sampled): where
    pi^-1 of Sec. III-D is defined."""
    th = np.linspace(0.0, calib.theta_max, samples)
    return bool(np.all(np.diff(radial(calib, th)) > 0.0))

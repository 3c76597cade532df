"""Trajectory field, calibration field / pre-rotation, triangulation (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

Conventions: a pose (R, t) maps camera-0 coordinates to camera-1 coordinates,
X1 = R X0 + t (the exp(xi_1) . X of Sec. III-A).  After the pre-rotation of
Sec. IV-A the second image is seen by a *virtual* camera with camera 0's
orientation and intrinsics, so the rig becomes a pure translation
X1' = X0 + t' with t' = R^T t, and the virtual camera's centre is C = -t'.
"""
from __future__ import annotations

import numpy as np

from .camera import project, unproject
from .interp import bilinear

SMALL_MOTION = 1e-5       # |t| -> 0 of Sec. III-B, Eq. 7 (symmetric pair, O(s^2) error)
EPIPOLE_RATIO = 1e-3      # |w| / s below this: the pixel is an epipole, gamma' = 0


def virtual_translation(R, t):
    """t' = R^T t: translation of the pre-rotated pair (Sec. IV-A)."""
    R = np.asarray(R, dtype=np.float64).reshape(3, 3)
    t = np.asarray(t, dtype=np.float64).reshape(3)
    return R.T @ t


def trajectory_vector(calib, tprime, px, py, depth=1.0, s=SMALL_MOTION):
    """gamma'(x0) at arbitrary points, following Sec. III-B.

    A surface point X at arbitrary depth on the ray of x0 is projected into
    cameras translated along t' by a vanishing amount (Eq. 6-7, |t| -> 0);
    the normalised flow w/|w| is the field.  The limit is taken with the
    symmetric pair of motions -s t'/|t'| and +s t'/|t'|, whose flow
    w = pi(X + s t^) - pi(X - s t^) has an O(s^2) error (a one-sided pair
    has O(s), about 1e-6 in gamma' for s = 1e-6, which the warping then
    amplifies).  Where |w|/(2 s) is below EPIPOLE_RATIO the point is an
    epipole and the field is 0.
    """
    tprime = np.asarray(tprime, dtype=np.float64)
    that = tprime / np.linalg.norm(tprime)
    X = depth * unproject(calib, px, py)
    x1 = project(calib, X + s * that)
    xm = project(calib, X - s * that)
    w = x1 - xm
    n = np.linalg.norm(w, axis=-1, keepdims=True)
    ok = n / (2.0 * s) >= EPIPOLE_RATIO
    return np.where(ok, w / np.where(ok, n, 1.0), 0.0)


def trajectory_field(calib, tprime, W, H, mask):
    """Trajectory field (H, W, 2) of one pyramid level; 0 outside the mask
    (Sec. III-B, Eq. 6-7)."""
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    g = trajectory_vector(calib, tprime, px, py)
    return np.where(mask[..., None], g, 0.0)


def calibration_field(calib0, calib1, R, W, H, mask0, depth=1.0):
    """Calibration field c(x) = pi_1(R X) - pi_0(X), t = 0 (Sec. IV-A); 0 off-mask."""
    R = np.asarray(R, dtype=np.float64).reshape(3, 3)
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    X = depth * unproject(calib0, px, py)
    x0 = project(calib0, X)
    x1 = project(calib1, X @ R.T)
    return np.where(mask0[..., None], x1 - x0, 0.0)


def prerotate(I1, cfield):
    """I1'(x) = I1(x + c(x)), bilinear (Sec. IV-A: warp the second image once)."""
    H, W = I1.shape
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    return bilinear(I1, px + cfield[..., 0], py + cfield[..., 1])


def triangulate_range(calib, px, py, wx, wy, tprime):
    """Range along the camera-0 ray of x, triangulated with the ray of x + w
    (Sec. III-D).

    Least-squares midpoint of the lines l0 * r0 and C + l1 * r1 with unit
    rays r0 = pi^-1(x), r1 = pi^-1(x + w) and the virtual camera-1 centre
    C = -t'.  Returns l0 (the distance from camera 0 along r0); +inf where
    the rays are parallel.  Written as the 2x2 normal equations.
    """
    r0 = unproject(calib, px, py)
    r1 = unproject(calib, np.asarray(px) + wx, np.asarray(py) + wy)
    C = -np.asarray(tprime, dtype=np.float64)
    b = np.sum(r0 * r1, axis=-1)
    d0 = r0 @ C
    d1 = r1 @ C
    # normal equations [[1, -b], [b, -1]] [l0, l1] = [d0, d1]; their
    # determinant 1 - b^2 equals |r0 x r1|^2 for unit rays, taken in that form
    det = np.sum(np.cross(r0, r1) ** 2, axis=-1)
    par = det <= 1e-24
    l0 = (d0 - b * d1) / np.where(par, 1.0, det)
    return np.where(par, np.inf, l0)

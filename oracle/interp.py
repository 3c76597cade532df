"""Image sampling at real-valued positions in float64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

* bilinear: the warp of I1 along w (Eq. 9, "Warp I1 using w" in Algorithm 1).
* bicubic: the trajectory field at the warped point (Sec. III-B: the tangent
  at the next warping step is read off the field by bicubic interpolation).
  Keys cubic convolution with a = -0.5.

Both clamp the sample position to [0, W-1] x [0, H-1] before sampling, so the
sampled value is a continuous function of the position everywhere; bicubic
taps that fall off the image repeat the edge pixel.  Arrays are (H, W) with
x the column and y the row; pixel centres are at integer coordinates.
"""
from __future__ import annotations

import numpy as np

KEYS_A = -0.5


def _clamp_pos(v, n):
    """Sample positions clamped to the image: the clamp-to-edge sampling of
    the warp (Eq. 9) and of the trajectory field (Sec. III-B)."""
    return np.clip(np.asarray(v, dtype=np.float64), 0.0, float(n - 1))


def bilinear(img, x, y):
    """Bilinear sample of img (H, W[, C]) at positions x, y (same shape): the
    warp of I1 along w (Eq. 9, Sec. III-C)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape[:2]
    xc = _clamp_pos(x, W)
    yc = _clamp_pos(y, H)
    x0 = np.minimum(np.floor(xc), max(W - 2, 0)).astype(np.int64)
    y0 = np.minimum(np.floor(yc), max(H - 2, 0)).astype(np.int64)
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    ax = xc - x0
    ay = yc - y0
    if img.ndim == 3:
        ax = ax[..., None]
        ay = ay[..., None]
    return ((1.0 - ax) * (1.0 - ay) * img[y0, x0] + ax * (1.0 - ay) * img[y0, x1]
            + (1.0 - ax) * ay * img[y1, x0] + ax * ay * img[y1, x1])


def keys_weight(s, a: float = KEYS_A):
    """Keys (1981) cubic convolution kernel, for the bicubic interpolation of
    the trajectory field (Sec. III-B)."""
    s = np.abs(np.asarray(s, dtype=np.float64))
    w_in = ((a + 2.0) * s - (a + 3.0)) * s * s + 1.0
    w_out = ((a * s - 5.0 * a) * s + 8.0 * a) * s - 4.0 * a
    return np.where(s <= 1.0, w_in, np.where(s < 2.0, w_out, 0.0))


def bicubic(img, x, y):
    """Keys-bicubic sample of img (H, W[, C]) at positions x, y: the trajectory
    field read at x + w (Sec. III-B)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape[:2]
    xc = _clamp_pos(x, W)
    yc = _clamp_pos(y, H)
    xi = np.floor(xc).astype(np.int64)
    yi = np.floor(yc).astype(np.int64)
    out = 0.0
    for j in range(-1, 3):
        yy = np.clip(yi + j, 0, H - 1)
        wy = keys_weight(yc - (yi + j))
        row = 0.0
        for i in range(-1, 3):
            xx = np.clip(xi + i, 0, W - 1)
            wx = keys_weight(xc - (xi + i))
            if img.ndim == 3:
                row = row + wx[..., None] * img[yy, xx]
            else:
                row = row + wx * img[yy, xx]
        out = out + (wy[..., None] * row if img.ndim == 3 else wy * row)
    return out

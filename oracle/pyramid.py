"""Coarse-to-fine pyramid and circular FOV mask (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

Sec. IV-B: the method runs N warps per level from coarse to fine and carries
disparity u and warp vector w up to the next level; a circular mask rejects
pixels beyond the desired FOV, Neumann/Dirichlet conditions are applied on
it, and it follows the image down the pyramid.  Sec. IV-C: scale factor 2.

Readings used here:
* level l has size ceil(W / 2^l) x ceil(H / 2^l); its calibration is the
  continuous rescaling f_l = f 2^-l, c_l = (c + 0.5) 2^-l - 0.5;
* the mask of level l is recomputed from that calibration
  (|m| <= r(theta_max)), the exact counterpart of a nearest-neighbour rescale;
* downsampling is the 2x2 box mean over the children inside the finer mask
  (all existing children when none is inside);
* upsampling is bilinear over the coarse in-mask samples with weights
  renormalised, values multiplied by 2 (disparity in pixels doubles), and 0
  outside the fine mask.
"""
from __future__ import annotations

import numpy as np

from .camera import Calib, radial


def level_sizes(W, H, levels):
    """Level sizes of the coarse-to-fine pyramid at scale 0.5 (Sec. IV-B)."""
    sizes = [(int(W), int(H))]
    for _ in range(1, levels):
        w, h = sizes[-1]
        sizes.append(((w + 1) // 2, (h + 1) // 2))
    return sizes


def scaled_calib(calib: Calib, level: int) -> Calib:
    """Calibration of pyramid level `level`: focal lengths and principal
    point scaled by 2^-level about pixel centres (Sec. IV-B)."""
    s = 0.5 ** level
    return Calib(calib.model, calib.fx * s, calib.fy * s,
                 (calib.cx + 0.5) * s - 0.5, (calib.cy + 0.5) * s - 0.5,
                 calib.k, calib.fov_deg)


def fov_mask(calib: Calib, W, H):
    """Pixels whose ray lies within the FOV half-angle (bool, (H, W)): the
    mask of each pyramid level (Sec. IV-B)."""
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    rn = np.hypot((px - calib.cx) / calib.fx, (py - calib.cy) / calib.fy)
    return rn <= float(radial(calib, calib.theta_max))


def downsample(img, mask_fine, Wc, Hc):
    """2x2 box mean over in-mask children (all children if none is in mask):
    one pyramid step (Sec. IV-B)."""
    img = np.asarray(img, dtype=np.float64)
    Hf, Wf = img.shape
    out = np.zeros((Hc, Wc))
    for Y in range(Hc):
        for X in range(Wc):
            kids = [(2 * Y + j, 2 * X + i) for j in (0, 1) for i in (0, 1)
                    if 2 * Y + j < Hf and 2 * X + i < Wf]
            inm = [k for k in kids if mask_fine[k]]
            use = inm if inm else kids
            out[Y, X] = sum(img[k] for k in use) / len(use)
    return out


def downsample_fast(img, mask_fine, Wc, Hc):
    """Vectorised twin of :func:`downsample` (same arithmetic per parent; one
    pyramid step of Sec. IV-B)."""
    img = np.asarray(img, dtype=np.float64)
    Hf, Wf = img.shape
    s_in = np.zeros((Hc, Wc)); n_in = np.zeros((Hc, Wc))
    s_all = np.zeros((Hc, Wc)); n_all = np.zeros((Hc, Wc))
    for j in (0, 1):
        for i in (0, 1):
            ys = 2 * np.arange(Hc) + j
            xs = 2 * np.arange(Wc) + i
            vy = ys < Hf
            vx = xs < Wf
            ex = np.outer(vy, vx)
            yy = np.minimum(ys, Hf - 1)
            xx = np.minimum(xs, Wf - 1)
            v = img[np.ix_(yy, xx)]
            m = mask_fine[np.ix_(yy, xx)] & ex
            s_all += np.where(ex, v, 0.0); n_all += ex
            s_in += np.where(m, v, 0.0); n_in += m
    return np.where(n_in > 0, s_in / np.maximum(n_in, 1), s_all / np.maximum(n_all, 1))


def upsample(v, mask_c, Wf, Hf, mask_f, scale=2.0):
    """Masked bilinear x2 upsampling of a (Hc, Wc[, C]) field to (Hf, Wf[, C]):
    u and w carried to the next finer level and doubled (Sec. IV-B)."""
    v = np.asarray(v, dtype=np.float64)
    Hc, Wc = v.shape[:2]
    py, px = np.mgrid[0:Hf, 0:Wf].astype(np.float64)
    X = np.clip((px + 0.5) * 0.5 - 0.5, 0.0, Wc - 1.0)
    Y = np.clip((py + 0.5) * 0.5 - 0.5, 0.0, Hc - 1.0)
    x0 = np.minimum(np.floor(X), max(Wc - 2, 0)).astype(np.int64)
    y0 = np.minimum(np.floor(Y), max(Hc - 2, 0)).astype(np.int64)
    x1 = np.minimum(x0 + 1, Wc - 1)
    y1 = np.minimum(y0 + 1, Hc - 1)
    ax = X - x0
    ay = Y - y0
    taps = [((1 - ax) * (1 - ay), y0, x0), (ax * (1 - ay), y0, x1),
            ((1 - ax) * ay, y1, x0), (ax * ay, y1, x1)]
    num = 0.0
    den = 0.0
    for wgt, yy, xx in taps:
        wm = wgt * mask_c[yy, xx]
        den = den + wm
        num = num + (wm[..., None] * v[yy, xx] if v.ndim == 3 else wm * v[yy, xx])
    if v.ndim == 3:
        out = np.where(den[..., None] > 0, num / np.where(den > 0, den, 1.0)[..., None], 0.0)
        return np.where(mask_f[..., None], scale * out, 0.0)
    out = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return np.where(mask_f, scale * out, 0.0)

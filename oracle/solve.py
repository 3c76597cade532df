"""Algorithm 1, coarse to fine, in float64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

Order of operations (Algorithm 1 inside the pyramid of Sec. IV-B, after the
pre-rotation of Sec. IV-A):

  pre-rotate I1 by the calibration field (t = 0)            Sec. IV-A
  build the image pyramids and the per-level masks          Sec. IV-B
  for each level, coarsest first:
      trajectory field gamma' of the level                  Sec. III-B
      tensor T^1/2 and step sizes                           Eq. 12, 11
      u, w <- 2 x upsampled previous level (0 at the top); p <- 0
      for each warp omega < N:
          warp I1 by w, linearise along gamma'              Eq. 3, 5, 9
          ubar <- u;  nIters primal-dual iterations          Eq. 11, 13
          clip delta-u, u_{w+1} = u_w + du, w += du g        Eq. 8, 9
  triangulate x and x + w at full resolution                Sec. III-D

The dual p carries over between the warps of one level and restarts at 0 on
a new level.  All state is float64.
"""
from __future__ import annotations

import numpy as np

from .camera import calib_from_dict
from .geometry import (calibration_field, prerotate, trajectory_field,
                       triangulate_range, virtual_translation)
from .pyramid import downsample_fast, fov_mask, level_sizes, scaled_calib, upsample
from .interp import bicubic
from .tgv import tgv_iteration, tgv_steps
from .variational import (Params, check_accel, clip_update, grad_masks, pd_iteration,
                          precondition, tensor_sqrt, warp_linearize)


def level_data(I0l, M, prm: Params):
    """Per-level constants: T^1/2 (Eq. 12), the gradient masks and the
    diagonal steps of the primal-dual iterations (Sec. III-D)."""
    a, b, c = tensor_sqrt(I0l, M, prm.beta, prm.eta)
    m1, m2 = grad_masks(M)
    tau, sig1, sig2 = precondition(a, b, c, M, m1, m2, prm.precond)
    lv = dict(a=a, b=b, c=c, m1=m1, m2=m2, M=M, tau=tau, sig1=sig1, sig2=sig2)
    if prm.regularizer == "tgv":
        lv["tau_u"], lv["tau_v"], lv["sig_p"], lv["sig_q"] = tgv_steps(a, b, c, M, m1, m2,
                                                                        prm.precond)
    return lv


TGV_STATE = ("v1", "v2", "q11", "q12", "q21", "q22")


def tgv_zero_state(shape):
    """v and q of a new level: 0 (like p, Sec. III-C state across levels)."""
    return {k: np.zeros(shape) for k in TGV_STATE}


def solve_level_warps(I0l, I1l, gamma, lv, u, w, p1, p2, warps, iters,
                      prm: Params, on_iter=None, level=0, tgv=None):
    """Run `warps` warps of `iters` primal-dual iterations on one level
    (Algorithm 1).

    tgv: for the TGV-L1 energy, the dict of v and q (TGV_STATE), carried
    across the warps like p and updated in place."""
    M = lv["M"]
    for om in range(warps):
        Iu, rho0, g = warp_linearize(I0l, I1l, w, gamma, M, prm.deriv)
        st = dict(u=u.copy(), ubar=u.copy(), p1=p1, p2=p2, Iu=Iu, rho0=rho0,
                  u_w=u.copy(), k=0)
        if tgv is not None:
            st.update(tgv, vb1=tgv["v1"].copy(), vb2=tgv["v2"].copy())
        if on_iter is not None:
            on_iter(level, om, -1, st, lv)
        for k in range(iters):
            if tgv is not None:
                tgv_iteration(st, lv, prm)
            else:
                pd_iteration(st, lv, prm)
            if on_iter is not None:
                on_iter(level, om, k, st, lv)
        u, w = clip_update(st["u"], st["u_w"], w, g, prm.du_max, M)
        p1, p2 = st["p1"], st["p2"]
        if tgv is not None:
            tgv.update({k: st[k] for k in TGV_STATE})
    return u, w, p1, p2


def warm_start_w(d, gamma, M, du_max):
    """Warp vector of a given disparity d: walk along the trajectory field
    from x in n = ceil(|d| / du_max) equal steps of d / n, each along the
    renormalised bicubic gamma' at the current point (the update w += du g of
    Algorithm 1 repeated with the largest admissible increments).  n is
    taken in float32, the precision of the stored disparity."""
    H, W = d.shape
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    n = np.ceil(np.float32(np.abs(d)) / np.float32(du_max)).astype(np.int64)
    n = np.where(M, n, 0)
    step = np.where(n > 0, d / np.maximum(n, 1), 0.0)
    w = np.zeros((H, W, 2))
    for k in range(int(n.max()) if n.size else 0):
        act = n > k
        graw = bicubic(gamma, px + w[..., 0], py + w[..., 1])
        nrm = np.hypot(graw[..., 0], graw[..., 1])
        ok = act & (nrm >= 1e-6)
        g = np.where(ok[..., None], graw / np.where(ok, nrm, 1.0)[..., None], 0.0)
        w = w + step[..., None] * g
    return w


def solve(I0, I1, cam0, cam1, R, t, levels, warps, iters, prm: Params = Params(),
          on_iter=None, keep_levels=False, level_hook=None, d_init=None, w_init=None):
    """Full method on one pair; returns disparity (px), range (m), w and more:
    Algorithm 1 inside the pre-rotation of Sec. IV-A and the coarse-to-fine
    scheme of Sec. IV-B, then the triangulation of Sec. III-D.

    level_hook(level, I0_l, I1_l) -> (I0_l, I1_l), when given, may replace
    each level's images after the pyramid is built (a probe for how the
    result responds to perturbing them; None for the method itself).

    d_init, when given, warm-starts from that full-resolution disparity:
    u = d_init, w rebuilt by warm_start_w, and only the finest level runs.
    w_init (H, W, 2), given with d_init, is a video stream's continuation:
    w is taken as given (the previous frame's w) instead of being rebuilt.
    """
    check_accel(prm)
    cam0 = calib_from_dict(cam0)
    cam1 = calib_from_dict(cam1)
    I0 = np.asarray(I0, dtype=np.float64)
    I1 = np.asarray(I1, dtype=np.float64)
    H, W = I0.shape
    M0 = fov_mask(cam0, W, H)
    cfield = calibration_field(cam0, cam1, R, W, H, M0)
    I1p = prerotate(I1, cfield)
    tp = virtual_translation(R, t)

    sizes = level_sizes(W, H, levels)
    calibs = [scaled_calib(cam0, l) for l in range(levels)]
    masks = [fov_mask(calibs[l], *sizes[l]) for l in range(levels)]
    pyr0, pyr1 = [I0], [I1p]
    for l in range(1, levels):
        pyr0.append(downsample_fast(pyr0[-1], masks[l - 1], *sizes[l]))
        pyr1.append(downsample_fast(pyr1[-1], masks[l - 1], *sizes[l]))

    if level_hook is not None:
        for l in range(levels):
            pyr0[l], pyr1[l] = level_hook(l, pyr0[l], pyr1[l])

    u = w = None
    per_level = []
    first = levels - 1
    if d_init is not None:
        M = masks[0]
        gamma0 = trajectory_field(calibs[0], tp, W, H, M)
        u = np.where(M, np.asarray(d_init, dtype=np.float64), 0.0)
        if w_init is None:
            w = np.where(M[..., None], warm_start_w(u, gamma0, M, prm.du_max), 0.0)
        else:
            w = np.where(M[..., None], np.asarray(w_init, dtype=np.float64), 0.0)
        first = 0
    for l in range(first, -1, -1):
        Wl, Hl = sizes[l]
        M = masks[l]
        gamma = trajectory_field(calibs[l], tp, Wl, Hl, M)
        lv = level_data(pyr0[l], M, prm)
        if u is None:
            u = np.zeros((Hl, Wl))
            w = np.zeros((Hl, Wl, 2))
        elif l < first:
            u = upsample(u, masks[l + 1], Wl, Hl, M)
            w = upsample(w, masks[l + 1], Wl, Hl, M)
        p1 = np.zeros((Hl, Wl))
        p2 = np.zeros((Hl, Wl))
        tgv = tgv_zero_state((Hl, Wl)) if prm.regularizer == "tgv" else None
        u, w, p1, p2 = solve_level_warps(pyr0[l], pyr1[l], gamma, lv, u, w, p1, p2,
                                         warps, iters, prm, on_iter, l, tgv)
        if keep_levels:
            per_level.append(dict(level=l, u=u.copy(), w=w.copy(), gamma=gamma,
                                  I0=pyr0[l], I1=pyr1[l], **lv))

    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    rng = triangulate_range(cam0, px, py, w[..., 0], w[..., 1], tp)
    depth = np.where(M0, rng, np.nan)
    out = dict(disp=np.where(M0, u, 0.0), depth=depth, w=w, mask=M0, I1p=I1p,
               cfield=cfield, tprime=tp)
    if keep_levels:
        out["levels"] = per_level
    return out

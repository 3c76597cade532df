"""Tensor-weighted Huber-TV-L1 primal-dual step and linearisation (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

Energy (first-order member of the Eq. 10 family, with v = 0, alpha_1 = 1 and
a Huber norm on the regulariser):

    E_w(u) = sum_{x in M} lam |rho_bar(x, u)| + sum_x h_eps(T^1/2(x) grad u(x))
    rho_bar(x, u) = rho0(x) + I_u(x) (u(x) - u_w(x))              (Eq. 3, 5)
    h_eps(z) = |z|^2 / (2 eps) if |z| <= eps else |z| - eps / 2

K = T^1/2 grad.  One primal-dual iteration (Eq. 11 with the Huber resolvent
on the dual, Eq. 13 on the primal):

    p   <- P((p + sigma * K ubar) / (1 + sigma * eps)),  P(q) = q / max(1, |q|)
    uh  <- u + tau * div(T^1/2 p)
    u'  <- shrink(uh)                                      (Eq. 13, sign fixed)
    ubar <- u' + theta (u' - u)

Discretisation (Sec. IV-B boundary conditions on the mask M):
* grad uses forward differences; component c at x is 0 unless x and x + e_c
  are both inside the image and the mask (Neumann);
* div is the exact negative adjoint of that grad;
* u is only updated on M and stays 0 elsewhere (Dirichlet).

Step sizes (Pock & Chambolle 2011 diagonal preconditioning, alpha = 1): row
and column sums of the entrywise bound |T^1/2| |grad| >= |K|:
    sigma(x) = 1 / max_c (2 sum_d |T_cd(x)| m_d(x))      (shared by p1, p2)
    tau(x)   = 1 / ((|a|+|b|)(x) m1(x) + (|b|+|c|)(x) m2(x)
                    + (|a|+|b|)(x-e1) m1(x-e1) + (|b|+|c|)(x-e2) m2(x-e2))
(0 where the sum is 0); precond=False uses tau = sigma = 1/sqrt(8).
A separate sigma per component would make the radial projection P the wrong
resolvent (the fixed point is then not a minimiser of E), so both components
of p(x) take the smaller of the two row-sum bounds.
Arrays are (H, W); axis 1 is x (e1), axis 0 is y (e2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .interp import bicubic, bilinear


@dataclass(frozen=True)
class Params:
    lam: float = 50.0        # data weight (not stated in the paper; workload value)
    eps: float = 0.01        # Huber width (not in the paper; workload value)
    du_max: float = 0.2      # Sec. IV-C / Sec. V-A: delta-u clip, 0.2 px
    beta: float = 9.0        # Sec. IV-C, Eq. 12
    eta: float = 0.85        # Sec. IV-C, Eq. 12
    theta: float = 1.0       # over-relaxation (Chambolle-Pock Algorithm 1)
    precond: bool = True     # diagonal preconditioning (Pock-Chambolle 2011)
    regularizer: str = "huber_tv"   # or "tgv": the TGV-L1 energy of Eq. 10
    alpha0: float = 17.0     # Sec. IV-C, TGV second-order weight
    alpha1: float = 1.2      # Sec. IV-C, TGV first-order weight
    deriv: str = "forward"   # I_u: "forward" = Eq. 7; "central" = half the
                             # difference of the samples at x + w +- g
    accel_gamma: float = 0.0  # > 0: the step schedule of Chambolle-Pock's
                              # Algorithm 2 (Sec. IV-C's "theta updated every
                              # iteration"); scalar steps only (precond False)


def grad_masks(M):
    """Neumann masks m1, m2: forward difference along x / y is inside M (the
    discrete gradient of Eq. 11)."""
    M = np.asarray(M, dtype=bool)
    m1 = np.zeros_like(M)
    m2 = np.zeros_like(M)
    m1[:, :-1] = M[:, :-1] & M[:, 1:]
    m2[:-1, :] = M[:-1, :] & M[1:, :]
    return m1, m2


def grad(u, m1, m2):
    """Masked forward-difference gradient (g1 along x, g2 along y) of Eq. 11."""
    g1 = np.zeros_like(u, dtype=np.float64)
    g2 = np.zeros_like(u, dtype=np.float64)
    g1[:, :-1] = u[:, 1:] - u[:, :-1]
    g2[:-1, :] = u[1:, :] - u[:-1, :]
    return np.where(m1, g1, 0.0), np.where(m2, g2, 0.0)


def div(q1, q2, m1, m2):
    """Exact negative adjoint of :func:`grad`: <grad u, q> = -<u, div q>, the
    divergence of Eq. 11."""
    a = np.where(m1, q1, 0.0)
    b = np.where(m2, q2, 0.0)
    d = a + b
    d[:, 1:] -= a[:, :-1]
    d[1:, :] -= b[:-1, :]
    return d


def tensor_sqrt(I0, M, beta, eta):
    """T^1/2 = exp(-beta |grad I0|^eta) n n^T + n_perp n_perp^T   (Eq. 12).

    grad I0 by central differences on the masked image, one-sided where one
    neighbour leaves the mask, 0 where both do.  Returns the three distinct
    entries (a, b, c) of the symmetric matrix [[a, b], [b, c]]; identity
    outside the mask.
    """
    I0 = np.asarray(I0, dtype=np.float64)
    M = np.asarray(M, dtype=bool)
    H, W = I0.shape

    def central(axis):
        n = I0.shape[axis]
        fwd = np.zeros_like(I0)
        bwd = np.zeros_like(I0)
        mf = np.zeros_like(M)
        mb = np.zeros_like(M)
        if axis == 1:
            fwd[:, :-1] = I0[:, 1:] - I0[:, :-1]
            bwd[:, 1:] = I0[:, 1:] - I0[:, :-1]
            mf[:, :-1] = M[:, 1:]
            mb[:, 1:] = M[:, :-1]
        else:
            fwd[:-1, :] = I0[1:, :] - I0[:-1, :]
            bwd[1:, :] = I0[1:, :] - I0[:-1, :]
            mf[:-1, :] = M[1:, :]
            mb[1:, :] = M[:-1, :]
        return np.where(mf & mb, 0.5 * (fwd + bwd),
                        np.where(mf, fwd, np.where(mb, bwd, 0.0)))

    gx = central(1)
    gy = central(0)
    mag = np.hypot(gx, gy)
    big = mag >= 1e-12
    nx = np.where(big, gx / np.where(big, mag, 1.0), 1.0)
    ny = np.where(big, gy / np.where(big, mag, 1.0), 0.0)
    e = np.exp(-beta * mag ** eta)
    a = e * nx * nx + ny * ny
    b = (e - 1.0) * nx * ny
    c = e * ny * ny + nx * nx
    return (np.where(M, a, 1.0), np.where(M, b, 0.0), np.where(M, c, 1.0))


def precondition(a, b, c, M, m1, m2, precond=True):
    """Diagonal step sizes (tau, sigma1, sigma2) for K = T^1/2 grad: the
    preconditioning of Sec. III-D (Pock-Chambolle, alpha = 1)."""
    if not precond:
        s = 1.0 / np.sqrt(8.0)
        f = np.full(a.shape, s)
        return f.copy(), f.copy(), f.copy()
    aa, bb, cc = np.abs(a), np.abs(b), np.abs(c)
    r1 = 2.0 * (aa * m1 + bb * m2)
    r2 = 2.0 * (bb * m1 + cc * m2)
    col = (aa + bb) * m1 + (bb + cc) * m2
    left = (aa + bb) * m1
    up = (bb + cc) * m2
    col[:, 1:] += left[:, :-1]
    col[1:, :] += up[:-1, :]
    # one sigma for both components of p(x): the larger row sum bounds both,
    # and with equal weights P is the exact resolvent of the unit-ball constraint
    r = np.maximum(r1, r2)
    sig = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
    tau = np.where((col > 0) & M, 1.0 / np.where(col > 0, col, 1.0), 0.0)
    return tau, sig, sig.copy()


def apply_T(a, b, c, v1, v2):
    """T^1/2 = [[a, b], [b, c]] applied to the field (v1, v2) (Eq. 12)."""
    return a * v1 + b * v2, b * v1 + c * v2


def dual_step(p1, p2, ubar, a, b, c, m1, m2, sig1, sig2, eps):
    """Dual ascent with the Huber resolvent and the projection P (Eq. 11)."""
    g1, g2 = grad(ubar, m1, m2)
    k1, k2 = apply_T(a, b, c, g1, g2)
    q1 = (p1 + sig1 * k1) / (1.0 + sig1 * eps)
    q2 = (p2 + sig2 * k2) / (1.0 + sig2 * eps)
    n = np.maximum(1.0, np.hypot(q1, q2))
    return q1 / n, q2 / n


def shrink(uh, Iu, rho0, u_w, tau, lam):
    """Resolvent (I + tau dG)^-1 of G(u) = lam |rho0 + Iu (u - u_w)|  (Eq. 13).

    Eq. 13 prints the third case with +rho_bar/I_u; the minimiser of
    (u - uh)^2 / (2 tau) + lam |rho_bar(u)| has -rho_bar(uh)/I_u there.
    """
    r = rho0 + Iu * (uh - u_w)
    thr = tau * lam * Iu * Iu
    step = tau * lam * Iu
    inner = np.where(Iu != 0.0, -r / np.where(Iu != 0.0, Iu, 1.0), 0.0)
    return uh + np.where(r < -thr, step, np.where(r > thr, -step, inner))


def primal_step(u, p1, p2, a, b, c, m1, m2, tau, Iu, rho0, u_w, lam, M):
    """Primal descent u + tau div(T^1/2 p), then the pointwise shrinkage
    (Eq. 11, 13)."""
    q1, q2 = apply_T(a, b, c, p1, p2)
    uh = u + tau * div(q1, q2, m1, m2)
    return np.where(M, shrink(uh, Iu, rho0, u_w, tau, lam), u)


def accel_schedule(gamma, n, tau0=1.0 / np.sqrt(8.0), sig0=1.0 / np.sqrt(8.0)):
    """Steps of Chambolle-Pock's Algorithm 2 for n iterations: iteration k
    uses tau_k and sigma_k, relaxes with theta_k = 1 / sqrt(1 + 2 gamma tau_k),
    then tau_{k+1} = theta_k tau_k and sigma_{k+1} = sigma_k / theta_k.
    Returns arrays (tau, sigma, theta) of length n."""
    tau = np.empty(n)
    sig = np.empty(n)
    th = np.empty(n)
    t, s = tau0, sig0
    for k in range(n):
        tau[k], sig[k] = t, s
        th[k] = 1.0 / np.sqrt(1.0 + 2.0 * gamma * t)
        t, s = th[k] * t, s / th[k]
    return tau, sig, th


def check_accel(prm: Params):
    """The conditions of the accelerated step schedule (Sec. III-D's theta
    updated every iteration): finite gamma >= 0, scalar steps, Huber-TV."""
    if prm.accel_gamma < 0 or not np.isfinite(prm.accel_gamma):
        raise ValueError("accel_gamma must be finite and >= 0")
    if prm.accel_gamma > 0 and (prm.precond or prm.regularizer != "huber_tv"):
        raise ValueError("the accelerated schedule needs scalar steps (precond False) "
                         "and the Huber-TV regulariser")


def pd_iteration(st, lv, prm: Params):
    """One iteration of Eq. 11 on state dict st (u, ubar, p1, p2) with level
    data lv.

    With prm.accel_gamma > 0 the scalar steps and the relaxation follow
    accel_schedule, restarted at every warp: st["k"] counts the warp's
    iterations (solve_level_warps sets it to 0); tau_k applies on the mask
    only (u is held outside it) and sigma_k everywhere, as the unaccelerated
    scalar steps do."""
    if prm.accel_gamma > 0:
        k = st["k"]
        tau_s, sig_s, th_s = accel_schedule(prm.accel_gamma, k + 1)
        sig = np.full(lv["M"].shape, sig_s[k])
        tau = np.where(lv["M"], tau_s[k], 0.0)
        theta = th_s[k]
        st["k"] = k + 1
    else:
        sig, tau, theta = lv["sig1"], lv["tau"], prm.theta
    p1, p2 = dual_step(st["p1"], st["p2"], st["ubar"], lv["a"], lv["b"], lv["c"],
                       lv["m1"], lv["m2"], sig, sig if prm.accel_gamma > 0 else lv["sig2"],
                       prm.eps)
    u_new = primal_step(st["u"], p1, p2, lv["a"], lv["b"], lv["c"], lv["m1"], lv["m2"],
                        tau, st["Iu"], st["rho0"], st["u_w"], prm.lam, lv["M"])
    ubar = u_new + theta * (u_new - st["u"])
    st.update(u=u_new, ubar=ubar, p1=p1, p2=p2)
    return st


def warp_linearize(I0, I1, w, gamma, M, deriv="forward"):
    """Warp I1 along w and linearise along the trajectory (Eq. 3, 5, 9).

    g = bicubic gamma'(x + w) renormalised (0 when |g| < 1e-6);
    I1w = I1(x + w);  rho0 = I1w - I0;
    I_u = I1(x + w + g) - I1w                        deriv "forward" (Eq. 7)
    I_u = (I1(x + w + g) - I1(x + w - g)) / 2        deriv "central"
    The forward difference of Eq. 7 shares the sample I1w with rho0, so
    independent image noise of variance s^2 gives E[I_u rho0] a -s^2 term:
    each warp's step is biased towards +u.  The central difference does not
    contain I1w (no such term) and is exact on a quadratic image.
    Returns (Iu, rho0, g), all 0 outside the mask.
    """
    if deriv not in ("forward", "central"):
        raise ValueError(f"deriv must be 'forward' or 'central', not {deriv!r}")
    H, W = I0.shape
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    xs = px + w[..., 0]
    ys = py + w[..., 1]
    graw = bicubic(gamma, xs, ys)
    n = np.hypot(graw[..., 0], graw[..., 1])
    ok = n >= 1e-6
    g = np.where(ok[..., None], graw / np.where(ok, n, 1.0)[..., None], 0.0)
    I1w = bilinear(I1, xs, ys)
    I1g = bilinear(I1, xs + g[..., 0], ys + g[..., 1])
    if deriv == "forward":
        Iu = I1g - I1w
    else:
        Iu = 0.5 * (I1g - bilinear(I1, xs - g[..., 0], ys - g[..., 1]))
    Iu = np.where(M, Iu, 0.0)
    rho0 = np.where(M, I1w - I0, 0.0)
    return Iu, rho0, np.where(M[..., None], g, 0.0)


def clip_update(u, u_w, w, g, du_max, M):
    """Clip delta-u, advance u_w and w (Algorithm 1, Eq. 8-9)."""
    du = np.where(M, np.clip(u - u_w, -du_max, du_max), 0.0)
    u_next = u_w + du
    return u_next, w + du[..., None] * g


def huber(z1, z2, eps):
    """Huber norm h_eps of the first-order regulariser (Eq. 10 with v = 0)."""
    n = np.hypot(z1, z2)
    return np.where(n <= eps, n * n / (2.0 * eps), n - eps / 2.0)


def energy(u, u_w, Iu, rho0, a, b, c, m1, m2, M, lam, eps):
    """E_w(u) of the linearised problem of one warp (Eq. 10 with v = 0, the
    data term of Eq. 5)."""
    g1, g2 = grad(u, m1, m2)
    k1, k2 = apply_T(a, b, c, g1, g2)
    data = lam * np.abs(rho0 + Iu * (u - u_w))
    return float(np.sum(np.where(M, data, 0.0)) + np.sum(huber(k1, k2, eps)))

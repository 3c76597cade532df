"""Tensor-guided TGV-L1 primal-dual step (Sec. III-C, Eq. 10-11), FP64 oracle.

Test infrastructure only (see ``oracle/__init__``).

Energy of one warp (Eq. 10 with the linearised data term of Eq. 3, 5):

    E_w(u, v) = sum_{x in M} lam |rho_bar(x, u)|
              + alpha1 sum_x |T^1/2 grad u - v| + alpha0 sum_x |grad v|

with v = (v1, v2) a vector field and grad v its 2 x 2 Jacobian (q has four
components, Sec. III-C).  Saddle-point form with the operator
K(u, v) = (T^1/2 grad u - v, grad v) and duals p (2 per pixel), q (4):

    p    <- Pi_alpha1(p + sigma_p (T^1/2 grad ubar - vbar))
    q    <- Pi_alpha0(q + sigma_q grad vbar)
    u    <- shrink(u + tau_u div(T^1/2 p))                    (Eq. 13)
    v    <- v + tau_v (p + div q)
    ubar <- u' + theta (u' - u),  vbar <- v' + theta (v' - v)

Pi_r projects each pixel's vector onto the ball of radius r (Euclidean for
p, Frobenius for q).  Eq. 11 prints the unit-ball projection with alpha1
and alpha0 inside the dual steps but not in the primal ones; the form above
is the consistent saddle point of Eq. 10 (the printed one, with p scaled by
alpha1 and q by alpha0).  No Huber smoothing: the paper's TGV is plain L1.

Discretisation: grad and div are the masked forward differences and their
exact negative adjoint of :mod:`oracle.variational`, applied to each
component of v and each row of q; u and v are held at 0 outside the mask.

Step sizes (Pock & Chambolle 2011 diagonal preconditioning, alpha = 1, on
the entrywise bound of K):
    sigma_p(x) = 1 / (max_c rowsum_c(|T^1/2| |grad|)(x) + 1)   (shared by p1, p2)
    sigma_q(x) = 1 / 2                                        (shared by the four q)
    tau_u(x)   = the Huber-TV tau (column sum of |T^1/2| |grad|)
    tau_v(x)   = 1 / (1 + m1(x) + m1(x - e1) + m2(x) + m2(x - e2))
all 0 outside the mask; precond=False uses tau = sigma = 1/sqrt(12)
(|K|^2 <= 8 + 4 with |T^1/2| <= 1).
"""
from __future__ import annotations

import numpy as np

from .variational import apply_T, div, grad, precondition, shrink


def grad_v(v1, v2, m1, m2):
    """Jacobian of v: (dv1/dx, dv1/dy, dv2/dx, dv2/dy), masked forward differences
    (the second-order term of Eq. 10)."""
    a, b = grad(v1, m1, m2)
    c, d = grad(v2, m1, m2)
    return a, b, c, d


def div_q(q11, q12, q21, q22, m1, m2):
    """Exact negative adjoint of :func:`grad_v`: one divergence per row of q
    (Eq. 11)."""
    return div(q11, q12, m1, m2), div(q21, q22, m1, m2)


def tgv_steps(a, b, c, M, m1, m2, precond=True):
    """(tau_u, tau_v, sigma_p, sigma_q) for K(u, v) = (T^1/2 grad u - v, grad v):
    the preconditioned steps of Sec. III-D for Eq. 10-11."""
    M = np.asarray(M, dtype=bool)
    if not precond:
        s = 1.0 / np.sqrt(12.0)
        f = np.where(M, s, 0.0)
        return f.copy(), f.copy(), f.copy(), f.copy()
    tau_u, sig, _ = precondition(a, b, c, M, m1, m2, True)
    aa, bb, cc = np.abs(a), np.abs(b), np.abs(c)
    r = np.maximum(2.0 * (aa * m1 + bb * m2), 2.0 * (bb * m1 + cc * m2))
    sig_p = np.where(M, 1.0 / (r + 1.0), 0.0)
    sig_q = np.where(M, 0.5, 0.0)
    col = m1.astype(np.float64) + m2
    col[:, 1:] += m1[:, :-1]
    col[1:, :] += m2[:-1, :]
    tau_v = np.where(M, 1.0 / (1.0 + col), 0.0)
    return tau_u, tau_v, sig_p, sig_q


def _project(r, *comps):
    """Projection onto the ball of radius r (the dual constraints of Eq. 11)."""
    n = np.maximum(1.0, np.sqrt(sum(c * c for c in comps)) / r) if r > 0 else None
    if n is None:
        return tuple(np.zeros_like(c) for c in comps)
    return tuple(c / n for c in comps)


def tgv_iteration(st, lv, prm):
    """One iteration of Eq. 11 (TGV-L1) on state st (u, ubar, v1, v2, vb1, vb2,
    p1, p2, q11, q12,
    q21, q22, Iu, rho0, u_w) with level data lv (a, b, c, m1, m2, M and the
    TGV steps tau_u, tau_v, sig_p, sig_q)."""
    a, b, c, m1, m2, M = lv["a"], lv["b"], lv["c"], lv["m1"], lv["m2"], lv["M"]
    # dual ascent
    g1, g2 = grad(st["ubar"], m1, m2)
    k1, k2 = apply_T(a, b, c, g1, g2)
    sp = lv["sig_p"]
    p1, p2 = _project(prm.alpha1, st["p1"] + sp * (k1 - st["vb1"]),
                      st["p2"] + sp * (k2 - st["vb2"]))
    j = grad_v(st["vb1"], st["vb2"], m1, m2)
    sq = lv["sig_q"]
    q = _project(prm.alpha0, *(st[k] + sq * jk for k, jk in
                               zip(("q11", "q12", "q21", "q22"), j)))
    # primal descent
    t1, t2 = apply_T(a, b, c, p1, p2)
    uh = st["u"] + lv["tau_u"] * div(t1, t2, m1, m2)
    u = np.where(M, shrink(uh, st["Iu"], st["rho0"], st["u_w"], lv["tau_u"], prm.lam), st["u"])
    d1, d2 = div_q(*q, m1, m2)
    tv = lv["tau_v"]
    v1 = np.where(M, st["v1"] + tv * (p1 + d1), 0.0)
    v2 = np.where(M, st["v2"] + tv * (p2 + d2), 0.0)
    th = prm.theta
    st.update(ubar=u + th * (u - st["u"]), vb1=v1 + th * (v1 - st["v1"]),
              vb2=v2 + th * (v2 - st["v2"]), u=u, v1=v1, v2=v2, p1=p1, p2=p2,
              q11=q[0], q12=q[1], q21=q[2], q22=q[3])
    return st


def tgv_energy(u, v1, v2, u_w, Iu, rho0, a, b, c, m1, m2, M, lam, alpha0, alpha1):
    """E_w(u, v) of the linearised problem of one warp (Eq. 10)."""
    g1, g2 = grad(u, m1, m2)
    k1, k2 = apply_T(a, b, c, g1, g2)
    first = alpha1 * np.hypot(k1 - v1, k2 - v2)
    j = grad_v(v1, v2, m1, m2)
    second = alpha0 * np.sqrt(sum(x * x for x in j))
    data = lam * np.abs(rho0 + Iu * (u - u_w))
    return float(np.sum(np.where(M, data, 0.0)) + np.sum(np.where(M, first, 0.0))
                 + np.sum(second))

"""Pins for the oracle's tensor (Eq. 12), primal-dual step (Eq. 11, 13),
linearisation (Eq. 3, 5, 9) and energy."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle.interp import bicubic
from oracle.variational import (Params, apply_T, clip_update, div, dual_step, energy,
                                grad, grad_masks, pd_iteration, precondition, shrink,
                                tensor_sqrt, warp_linearize)


def _mask(H, W, seed):
    rng = np.random.default_rng(seed)
    M = rng.uniform(0, 1, (H, W)) > 0.15
    M[0, :] = True
    return M


def test_div_is_negative_adjoint_of_grad():
    rng = np.random.default_rng(0)
    for seed in range(3):
        H, W = 9 + seed, 13 - seed
        M = _mask(H, W, seed)
        m1, m2 = grad_masks(M)
        u = rng.normal(size=(H, W))
        q1 = rng.normal(size=(H, W))
        q2 = rng.normal(size=(H, W))
        g1, g2 = grad(u, m1, m2)
        lhs = np.sum(g1 * q1 + g2 * q2)
        rhs = -np.sum(u * div(q1, q2, m1, m2))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_grad_forward_difference_and_neumann():
    H, W = 6, 8
    py, px = np.mgrid[0:H, 0:W].astype(float)
    u = 2.0 * px - 3.0 * py
    M = np.ones((H, W), bool)
    M[3, 4] = False
    m1, m2 = grad_masks(M)
    g1, g2 = grad(u, m1, m2)
    assert g1[0, 0] == 2.0 and g2[0, 0] == -3.0
    assert np.all(g1[:, -1] == 0) and np.all(g2[-1, :] == 0)      # image edge
    assert g1[3, 3] == 0 and g1[3, 4] == 0 and g2[2, 4] == 0      # mask edge


def test_tensor_eigenstructure():
    rng = np.random.default_rng(1)
    H, W = 12, 12
    I0 = rng.uniform(0, 1, (H, W))
    M = np.ones((H, W), bool)
    beta, eta = 9.0, 0.85
    a, b, c = tensor_sqrt(I0, M, beta, eta)
    gy, gx = np.gradient(I0)               # central differences, one-sided at edges
    for y in range(1, H - 1):
        for x in range(1, W - 1):
            T = np.array([[a[y, x], b[y, x]], [b[y, x], c[y, x]]])
            g = np.array([gx[y, x], gy[y, x]])
            n = g / np.linalg.norm(g)
            e = np.exp(-beta * np.linalg.norm(g) ** eta)
            assert np.allclose(T @ n, e * n, atol=1e-13)
            assert np.allclose(T @ np.array([-n[1], n[0]]), [-n[1], n[0]], atol=1e-13)
    # flat image: identity
    a, b, c = tensor_sqrt(np.full((5, 5), 0.3), np.ones((5, 5), bool), beta, eta)
    assert np.all(a == 1.0) and np.all(b == 0.0) and np.all(c == 1.0)


def _dense_K(a, b, c, m1, m2):
    H, W = a.shape
    n = H * W
    K = np.zeros((2 * n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        g1, g2 = grad(e.reshape(H, W), m1, m2)
        k1, k2 = apply_T(a, b, c, g1, g2)
        K[:n, j] = k1.ravel()
        K[n:, j] = k2.ravel()
    return K


def test_preconditioned_steps_bound_the_operator():
    # Pock-Chambolle: || Sigma^1/2 K Tau^1/2 || <= 1
    rng = np.random.default_rng(2)
    H, W = 7, 9
    M = _mask(H, W, 4)
    a, b, c = tensor_sqrt(rng.uniform(0, 1, (H, W)), M, 9.0, 0.85)
    m1, m2 = grad_masks(M)
    tau, s1, s2 = precondition(a, b, c, M, m1, m2, True)
    K = _dense_K(a, b, c, m1, m2)
    S = np.sqrt(np.concatenate([s1.ravel(), s2.ravel()]))
    T = np.sqrt(tau.ravel())
    assert np.linalg.norm(S[:, None] * K * T[None, :], 2) <= 1.0 + 1e-12
    # tau is the reciprocal column sum of |T||grad| (brute force from matrices)
    n = H * W
    G = np.zeros((2 * n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        g1, g2 = grad(e.reshape(H, W), m1, m2)
        G[:n, j] = g1.ravel()
        G[n:, j] = g2.ravel()
    A = np.block([[np.diag(np.abs(a).ravel()), np.diag(np.abs(b).ravel())],
                  [np.diag(np.abs(b).ravel()), np.diag(np.abs(c).ravel())]])
    col = (A @ np.abs(G)).sum(axis=0)
    ref = np.where((col > 0) & M.ravel(), 1.0 / np.where(col > 0, col, 1), 0.0)
    assert np.allclose(tau.ravel(), ref, atol=1e-15)
    row = (A @ np.abs(G)).sum(axis=1)
    rmax = np.maximum(row[:n], row[n:])
    assert np.allclose(s1.ravel(), np.where(rmax > 0, 1 / np.where(rmax > 0, rmax, 1), 0))
    # scalar steps: tau sigma ||K||^2 <= 1
    t0, q0, _ = precondition(a, b, c, M, m1, m2, False)
    assert t0[0, 0] * q0[0, 0] * np.linalg.norm(K, 2) ** 2 <= 1.0 + 1e-12


def test_dual_step_is_huber_conjugate_prox():
    # with one sigma, p = argmin_{|p|<=1} eps/2 |p|^2 + |p - y|^2 / (2 sigma)
    rng = np.random.default_rng(3)
    eps = 0.05
    for _ in range(20):
        y = rng.normal(scale=1.5, size=2)
        sig = rng.uniform(0.05, 1.0)
        # dual_step with ubar = 0 and p = y gives the prox of y
        one = np.ones((1, 1), bool)
        p1, p2 = dual_step(np.array([[y[0]]]), np.array([[y[1]]]), np.zeros((1, 1)),
                           np.ones((1, 1)), np.zeros((1, 1)), np.ones((1, 1)), one, one,
                           np.array([[sig]]), np.array([[sig]]), eps)
        r = np.linspace(0, 1, 401)
        t = np.linspace(-np.pi, np.pi, 721)
        R, Tt = np.meshgrid(r, t)
        P = np.stack([R * np.cos(Tt), R * np.sin(Tt)], -1)
        obj = eps / 2 * np.sum(P * P, -1) + np.sum((P - y) ** 2, -1) / (2 * sig)
        best = P.reshape(-1, 2)[np.argmin(obj)]
        assert np.linalg.norm(np.array([p1[0, 0], p2[0, 0]]) - best) < 6e-3


def test_shrink_is_data_term_prox():
    rng = np.random.default_rng(4)
    lam = 3.0
    for _ in range(200):
        uh, Iu, rho0, uw = rng.normal(size=4) * np.array([2.0, 0.5, 0.4, 1.0])
        if rng.uniform() < 0.1:
            Iu = 0.0
        tau = rng.uniform(0.01, 1.0)
        f = lambda u: (u - uh) ** 2 / (2 * tau) + lam * abs(rho0 + Iu * (u - uw))
        ref = minimize_scalar(f, bounds=(uh - 10, uh + 10), method="bounded",
                              options=dict(xatol=1e-12)).x
        got = shrink(np.array(uh), np.array(Iu), np.array(rho0), np.array(uw),
                     np.array(tau), lam)
        assert f(float(got)) <= f(ref) + 1e-9
        assert abs(float(got) - ref) < 1e-5


def _level(H, W, seed, precond, lam, eps):
    rng = np.random.default_rng(seed)
    M = _mask(H, W, seed + 10)
    I0 = rng.uniform(0, 1, (H, W))
    prm = Params(lam=lam, eps=eps, precond=precond)
    a, b, c = tensor_sqrt(I0, M, prm.beta, prm.eta)
    m1, m2 = grad_masks(M)
    tau, s1, s2 = precondition(a, b, c, M, m1, m2, precond)
    lv = dict(a=a, b=b, c=c, m1=m1, m2=m2, M=M, tau=tau, sig1=s1, sig2=s2)
    Iu = np.where(M, rng.uniform(-0.5, 0.5, (H, W)), 0)
    rho0 = np.where(M, rng.uniform(-0.3, 0.3, (H, W)), 0)
    u0 = np.where(M, rng.uniform(-1, 1, (H, W)), 0)
    st = dict(u=u0.copy(), ubar=u0.copy(), p1=np.zeros((H, W)), p2=np.zeros((H, W)),
              Iu=Iu, rho0=rho0, u_w=u0.copy())
    return prm, lv, st


@pytest.mark.parametrize("precond", [True, False])
def test_pd_converges_to_energy_minimiser(precond):
    # optimality of E itself, written from its definition: p* = grad h_eps(K u*)
    # and div(T p*) in lam I_u d|.|(rho_bar(u*)) on every mask pixel
    prm, lv, st = _level(6, 7, 1, precond, lam=2.0, eps=0.1)
    for _ in range(12000):
        pd_iteration(st, lv, prm)
    u = st["u"]
    a, b, c, m1, m2, M = (lv[k] for k in ("a", "b", "c", "m1", "m2", "M"))
    g1, g2 = grad(u, m1, m2)
    k1, k2 = apply_T(a, b, c, g1, g2)
    nrm = np.hypot(k1, k2)
    s = np.where(nrm <= prm.eps, 1.0 / prm.eps, 1.0 / np.maximum(nrm, 1e-300))
    q1, q2 = apply_T(a, b, c, k1 * s, k2 * s)
    dv = div(q1, q2, m1, m2)
    r = st["rho0"] + st["Iu"] * (u - st["u_w"])
    lam, Iu = prm.lam, st["Iu"]
    off = np.abs(r) > 1e-9
    viol = np.where(off, np.abs(dv - lam * Iu * np.sign(r)),
                    np.maximum(0.0, np.abs(dv) - lam * np.abs(Iu)))
    assert viol[M].max() < 1e-6
    assert np.all(u[~M] == 0)


@pytest.mark.parametrize("seed", [2, 3])
def test_energy_descends_over_a_warp(seed):
    # Chambolle-Pock is not a descent method: early iterations may raise E
    # (up to ~1% on these cases).  What holds: the final energy is below the
    # start, E stops increasing once the iterates settle, and scalar and
    # preconditioned steps reach the same minimum.
    finals = []
    for precond in (False, True):
        prm, lv, st = _level(10, 12, seed, precond, lam=5.0, eps=0.05)
        args = lambda s: (s["u"], s["u_w"], s["Iu"], s["rho0"], lv["a"], lv["b"], lv["c"],
                          lv["m1"], lv["m2"], lv["M"], prm.lam, prm.eps)
        E = [energy(*args(st))]
        for _ in range(1500):
            pd_iteration(st, lv, prm)
            E.append(energy(*args(st)))
        E = np.array(E)
        assert E[-1] < 0.8 * E[0]
        assert np.all(np.diff(E[600:]) <= 1e-9 * E[0])
        assert E[-1] <= E.min() + 1e-9 * E[0]
        finals.append(E[-1])
    assert abs(finals[0] - finals[1]) <= 1e-6 * finals[0]


def test_accel_schedule_recursion():
    # Chambolle-Pock Algorithm 2: tau_k sigma_k stays tau_0 sigma_0, theta_k
    # lies in (0, 1], tau_k falls, and tau_k ~ 1 / (gamma k) for large k
    # (tau_{k+1}^-2 = tau_k^-2 + 2 gamma tau_k^-1 / (1 + ...) grows by about
    # 2 gamma / tau_k per step); gamma = 0 is the constant theta = 1 schedule
    from oracle import accel_schedule
    t0 = 1 / np.sqrt(8)
    tau, sig, th = accel_schedule(0.0, 50)
    assert np.all(tau == t0) and np.all(sig == t0) and np.all(th == 1.0)
    g = 0.3
    tau, sig, th = accel_schedule(g, 200000)
    assert np.allclose(tau * sig, t0 * t0, rtol=1e-12)
    assert np.all((th > 0) & (th <= 1)) and np.all(np.diff(tau) < 0)
    assert np.allclose(th, 1 / np.sqrt(1 + 2 * g * tau), rtol=1e-15)
    assert np.allclose(tau[1:], th[:-1] * tau[:-1], rtol=1e-15)
    k = np.arange(len(tau))
    assert abs(tau[-1] * g * k[-1] - 1.0) < 0.01


def test_accel_iteration_reduces_to_theta_one_and_settles():
    # gamma = 0 gives the plain scalar iteration bit for bit; gamma > 0 (an
    # accelerated schedule on a data term that is not uniformly convex, so
    # no rate is guaranteed) still lowers the energy and ends near the
    # minimum of the constant-step run
    finals = {}
    for gamma in (0.0, 1e-300, 0.05):
        prm, lv, st = _level(10, 12, 2, False, lam=5.0, eps=0.05)
        if gamma:
            prm = Params(lam=5.0, eps=0.05, precond=False, accel_gamma=gamma)
        st["k"] = 0
        args = lambda s: (s["u"], s["u_w"], s["Iu"], s["rho0"], lv["a"], lv["b"], lv["c"],
                          lv["m1"], lv["m2"], lv["M"], prm.lam, prm.eps)
        E0 = energy(*args(st))
        for _ in range(1500):
            pd_iteration(st, lv, prm)
        finals[gamma] = (energy(*args(st)), st["u"].copy())
        assert finals[gamma][0] < 0.8 * E0
    assert np.array_equal(finals[0.0][1], finals[1e-300][1])
    assert finals[0.05][0] <= finals[0.0][0] * (1 + 1e-3)
    with pytest.raises(ValueError):
        from oracle import check_accel
        check_accel(Params(accel_gamma=0.1, precond=True))


def test_warp_linearize_on_affine_image():
    # Eq. 5 equals Eq. 4 for an affine I1; rho0 = I1(x + w) - I0(x) exactly
    H, W = 16, 20
    py, px = np.mgrid[0:H, 0:W].astype(float)
    I1 = 0.2 + 0.01 * px + 0.02 * py
    rng = np.random.default_rng(5)
    I0 = rng.uniform(0, 1, (H, W))
    gam = np.zeros((H, W, 2))
    gam[..., 0] = 0.6
    gam[..., 1] = -0.8
    w = np.zeros((H, W, 2))
    w[..., 0] = 1.25
    w[..., 1] = 0.5
    M = np.zeros((H, W), bool)
    M[3:12, 3:14] = True
    Iu, rho0, g = warp_linearize(I0, I1, w, gam, M)
    assert np.allclose(g[M], [0.6, -0.8], atol=1e-14)
    assert np.allclose(Iu[M], 0.01 * 0.6 + 0.02 * -0.8, atol=1e-14)
    ref = 0.2 + 0.01 * (px + 1.25) + 0.02 * (py + 0.5) - I0
    assert np.allclose(rho0[M], ref[M], atol=1e-14)
    assert np.all(Iu[~M] == 0) and np.all(rho0[~M] == 0)


def test_warp_linearize_derivatives_on_quadratic_image():
    # I1 = q x^2 along gamma' = e1: the derivative at x + w is 2 q (x + w).
    # Bilinear sampling of a quadratic errs by q f (1 - f) at fraction f, the
    # same at x + w +- 1, so the central difference is exact and the forward
    # difference of Eq. 7 is off by the curvature term q (1 + 0 f).
    H, W = 8, 24
    py, px = np.mgrid[0:H, 0:W].astype(float)
    qc = 0.003
    I1 = qc * px * px
    I0 = np.zeros((H, W))
    gam = np.zeros((H, W, 2))
    gam[..., 0] = 1.0
    w = np.zeros((H, W, 2))
    w[..., 0] = 0.3
    M = np.zeros((H, W), bool)
    M[1:7, 2:20] = True
    exact = 2 * qc * (px + 0.3)
    Iu_f, rho_f, _ = warp_linearize(I0, I1, w, gam, M, "forward")
    Iu_c, rho_c, _ = warp_linearize(I0, I1, w, gam, M, "central")
    assert np.allclose(Iu_c[M], exact[M], atol=1e-13)
    assert np.allclose(Iu_f[M], exact[M] + qc, atol=1e-13)
    assert np.array_equal(rho_f, rho_c)
    with pytest.raises(ValueError):
        warp_linearize(I0, I1, w, gam, M, "backward")


def test_warp_linearize_renormalises_the_sampled_field():
    # a unit field that turns 0.9 rad per pixel: its bicubic sample half-way
    # between pixels is shorter than 1, and g is that sample renormalised to
    # unit length; on an affine I1 the forward I_u is then grad(I1) . g exactly
    H, W = 10, 24
    py, px = np.mgrid[0:H, 0:W].astype(float)
    phi = 0.9 * px
    gam = np.stack([np.cos(phi), np.sin(phi)], -1)
    I1 = 0.3 + 0.02 * px - 0.01 * py
    I0 = np.zeros((H, W))
    w = np.zeros((H, W, 2))
    w[..., 0] = 0.5
    M = np.zeros((H, W), bool)
    M[2:8, 2:20] = True
    Iu, rho0, g = warp_linearize(I0, I1, w, gam, M)
    raw = bicubic(gam, px + 0.5, py)
    assert np.hypot(raw[..., 0], raw[..., 1])[M].max() < 0.999     # the sample is short
    assert np.abs(np.hypot(g[..., 0], g[..., 1])[M] - 1.0).max() < 1e-12
    assert np.abs(Iu - (0.02 * g[..., 0] - 0.01 * g[..., 1]))[M].max() < 1e-13


def test_warp_linearize_noise_correlation():
    # I1 white noise of variance s^2, I0 independent, w = 0: the forward
    # difference shares I1(x) with rho0, so mean(I_u rho0) -> -s^2; the
    # central difference holds no I1(x) and the mean -> 0 (standard error
    # about s^2 sqrt(2) / sqrt(n))
    rng = np.random.default_rng(11)
    H, W = 256, 256
    s = 0.1
    I1 = rng.normal(0.0, s, (H, W))
    I0 = rng.normal(0.0, s, (H, W))
    gam = np.zeros((H, W, 2))
    gam[..., 1] = 1.0
    w = np.zeros((H, W, 2))
    M = np.zeros((H, W), bool)
    M[2:-2, 2:-2] = True
    n = M.sum()
    for deriv, want in (("forward", -s * s), ("central", 0.0)):
        Iu, rho0, _ = warp_linearize(I0, I1, w, gam, M, deriv)
        got = (Iu * rho0)[M].mean()
        assert abs(got - want) < 5 * s * s * np.sqrt(2.0 / n), (deriv, got)


def test_clip_update_cases():
    M = np.array([[True, True, True, False]])
    u = np.array([[0.5, -0.05, -1.0, 3.0]])
    uw = np.zeros((1, 4))
    w = np.zeros((1, 4, 2))
    g = np.tile(np.array([0.6, 0.8]), (1, 4, 1))
    un, wn = clip_update(u, uw, w, g, 0.2, M)
    assert np.allclose(un, [[0.2, -0.05, -0.2, 0.0]])
    assert np.allclose(wn[0, :, 0], [0.12, -0.03, -0.12, 0.0])
    assert np.allclose(wn[0, :, 1], [0.16, -0.04, -0.16, 0.0])

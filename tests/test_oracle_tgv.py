"""Pins for the oracle's TGV-L1 primal-dual step (Sec. III-C, Eq. 10-11).

Checked against what the mathematics fixes, not against retyped formulas:
the Jacobian / divergence pair is an exact adjoint pair; the preconditioned
steps satisfy the Pock-Chambolle bound on a dense matrix of the operator
built by applying it to unit vectors; with alpha0 = 0 the second-order term
lets v absorb any gradient, so the minimiser is the per-pixel zero of the
linearised residual; the fixed point satisfies the saddle-point optimality
conditions of Eq. 10 written from its definition; the energy settles to the
same minimum for scalar and preconditioned steps; and a rendered
fronto-parallel plane is recovered end to end.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.tgv import div_q, grad_v, tgv_energy, tgv_iteration, tgv_steps
from oracle.variational import Params, apply_T, div, grad, grad_masks, tensor_sqrt


def _mask(H, W, seed):
    rng = np.random.default_rng(seed)
    M = rng.uniform(0, 1, (H, W)) > 0.15
    M[0, :] = True
    return M


def test_jacobian_divergence_adjoint():
    rng = np.random.default_rng(0)
    for seed in range(3):
        H, W = 8 + seed, 11 - seed
        m1, m2 = grad_masks(_mask(H, W, seed))
        v1, v2 = rng.normal(size=(2, H, W))
        q = rng.normal(size=(4, H, W))
        j = grad_v(v1, v2, m1, m2)
        lhs = sum(np.sum(a * b) for a, b in zip(j, q))
        d1, d2 = div_q(*q, m1, m2)
        rhs = -np.sum(v1 * d1 + v2 * d2)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def _dense_K(a, b, c, m1, m2):
    """Matrix of K(u, v) = (T^1/2 grad u - v, grad v) from unit vectors."""
    H, W = a.shape
    n = H * W
    cols = []
    for j in range(3 * n):
        e = np.zeros(3 * n)
        e[j] = 1.0
        u, v1, v2 = e[:n].reshape(H, W), e[n:2 * n].reshape(H, W), e[2 * n:].reshape(H, W)
        g1, g2 = grad(u, m1, m2)
        k1, k2 = apply_T(a, b, c, g1, g2)
        jv = grad_v(v1, v2, m1, m2)
        cols.append(np.concatenate([(k1 - v1).ravel(), (k2 - v2).ravel()] +
                                   [x.ravel() for x in jv]))
    return np.stack(cols, 1)


def test_preconditioned_steps_bound_the_operator():
    rng = np.random.default_rng(3)
    H, W = 6, 8
    M = np.ones((H, W), bool)          # v and p live on the whole grid here
    a, b, c = tensor_sqrt(rng.uniform(0, 1, (H, W)), M, 9.0, 0.85)
    m1, m2 = grad_masks(M)
    K = _dense_K(a, b, c, m1, m2)
    tu, tv, sp, sq = tgv_steps(a, b, c, M, m1, m2, True)
    S = np.sqrt(np.concatenate([sp.ravel(), sp.ravel()] + [sq.ravel()] * 4))
    T = np.sqrt(np.concatenate([tu.ravel(), tv.ravel(), tv.ravel()]))
    assert np.linalg.norm(S[:, None] * K * T[None, :], 2) <= 1.0 + 1e-12
    # column sums of |K| give tau exactly for v; p rows give sigma_p
    col = np.abs(K).sum(axis=0)
    n = H * W
    assert np.allclose(tv.ravel(), 1.0 / col[n:2 * n]) and np.allclose(tv.ravel(), 1.0 / col[2 * n:])
    # sigma_p from the rows of the entrywise bound |T^1/2| |grad| (plus 1 for
    # the -v entry), the bound the Huber-TV steps use as well
    G = np.zeros((2 * n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        g1, g2 = grad(e.reshape(H, W), m1, m2)
        G[:n, j], G[n:, j] = g1.ravel(), g2.ravel()
    A = np.block([[np.diag(np.abs(a).ravel()), np.diag(np.abs(b).ravel())],
                  [np.diag(np.abs(b).ravel()), np.diag(np.abs(c).ravel())]])
    row = (A @ np.abs(G)).sum(axis=1) + 1.0
    assert np.allclose(sp.ravel(), 1.0 / np.maximum(row[:n], row[n:]))
    assert np.all(row <= np.abs(K[:2 * n]).sum(axis=1) * 2 + 1)
    t0, _, s0, _ = tgv_steps(a, b, c, M, m1, m2, False)
    assert t0[0, 0] * s0[0, 0] * np.linalg.norm(K, 2) ** 2 <= 1.0 + 1e-12


def _level(H, W, seed, precond, lam, alpha0=17.0, alpha1=1.2):
    rng = np.random.default_rng(seed)
    M = _mask(H, W, seed + 10)
    prm = Params(lam=lam, precond=precond, regularizer="tgv", alpha0=alpha0, alpha1=alpha1)
    a, b, c = tensor_sqrt(rng.uniform(0, 1, (H, W)), M, prm.beta, prm.eta)
    m1, m2 = grad_masks(M)
    tu, tv, sp, sq = tgv_steps(a, b, c, M, m1, m2, precond)
    lv = dict(a=a, b=b, c=c, m1=m1, m2=m2, M=M, tau_u=tu, tau_v=tv, sig_p=sp, sig_q=sq)
    Iu = np.where(M, rng.uniform(0.1, 0.5, (H, W)) * rng.choice([-1, 1], (H, W)), 0)
    rho0 = np.where(M, rng.uniform(-0.3, 0.3, (H, W)), 0)
    u0 = np.where(M, rng.uniform(-1, 1, (H, W)), 0)
    z = np.zeros((H, W))
    st = dict(u=u0.copy(), ubar=u0.copy(), Iu=Iu, rho0=rho0, u_w=u0.copy(),
              p1=z.copy(), p2=z.copy(), v1=z.copy(), v2=z.copy(), vb1=z.copy(), vb2=z.copy(),
              q11=z.copy(), q12=z.copy(), q21=z.copy(), q22=z.copy())
    return prm, lv, st


def test_free_second_order_term_leaves_the_data_minimiser():
    # alpha0 = 0: v can equal T^1/2 grad u at no cost, so every pixel sits at
    # the zero of rho0 + I_u (u - u_w), i.e. u = u_w - rho0 / I_u
    prm, lv, st = _level(7, 9, 4, True, lam=3.0, alpha0=0.0)
    for _ in range(6000):
        tgv_iteration(st, lv, prm)
    M = lv["M"]
    ref = st["u_w"] - st["rho0"] / np.where(M, st["Iu"], 1.0)
    assert np.abs(st["u"] - ref)[M].max() < 1e-6


@pytest.mark.parametrize("precond", [True, False])
@pytest.mark.parametrize("weights", [(17.0, 1.2, 2.0), (0.2, 0.5, 3.0)])
def test_fixed_point_satisfies_the_saddle_point_conditions(precond, weights):
    # the paper's (alpha0, alpha1) leave v constant (grad v = 0); the second
    # set makes grad v active, so both subgradient conditions are exercised
    # Eq. 10 optimality, from its definition: |p| <= alpha1 with
    # p = alpha1 (K1 u - v)/|K1 u - v| where K1 u - v != 0 (K1 = T^1/2 grad),
    # the same for q and grad v with alpha0, v-stationarity p + div q = 0,
    # and u-stationarity div(T^1/2 p) in lam I_u d|.|(rho_bar(u))
    a0, a1, lam = weights
    prm, lv, st = _level(6, 7, 1, precond, lam=lam, alpha0=a0, alpha1=a1)
    for _ in range(30000 if precond else 80000):      # the scalar steps are slower
        tgv_iteration(st, lv, prm)
    a, b, c, m1, m2, M = (lv[k] for k in ("a", "b", "c", "m1", "m2", "M"))
    u, v1, v2, p1, p2 = st["u"], st["v1"], st["v2"], st["p1"], st["p2"]
    q = [st[k] for k in ("q11", "q12", "q21", "q22")]
    g1, g2 = grad(u, m1, m2)
    k1, k2 = apply_T(a, b, c, g1, g2)
    r1, r2 = k1 - v1, k2 - v2
    nr = np.hypot(r1, r2)
    assert np.all(np.hypot(p1, p2) <= prm.alpha1 + 1e-9)
    big = M & (nr > 1e-3)
    assert big.sum() >= 4
    assert np.abs(p1 - prm.alpha1 * r1 / np.maximum(nr, 1e-300))[big].max() < 1e-4
    assert np.abs(p2 - prm.alpha1 * r2 / np.maximum(nr, 1e-300))[big].max() < 1e-4
    j = grad_v(v1, v2, m1, m2)
    nj = np.sqrt(sum(x * x for x in j))
    assert np.all(np.sqrt(sum(x * x for x in q)) <= prm.alpha0 + 1e-9)
    bigj = nj > 1e-3
    assert bigj.any() or a0 > 1.0
    for x, y in zip(q, j):
        if bigj.any():
            assert np.abs(x - prm.alpha0 * y / np.maximum(nj, 1e-300))[bigj].max() < 1e-4
    d1, d2 = div_q(*q, m1, m2)
    assert np.abs(p1 + d1)[M].max() < 1e-6 and np.abs(p2 + d2)[M].max() < 1e-6
    t1, t2 = apply_T(a, b, c, p1, p2)
    dv = div(t1, t2, m1, m2)
    rb = st["rho0"] + st["Iu"] * (u - st["u_w"])
    off = np.abs(rb) > 1e-9
    viol = np.where(off, np.abs(dv - prm.lam * st["Iu"] * np.sign(rb)),
                    np.maximum(0.0, np.abs(dv) - prm.lam * np.abs(st["Iu"])))
    assert viol[M].max() < 1e-5


def test_energy_settles_to_the_same_minimum_for_both_step_rules():
    finals = []
    for precond in (False, True):
        prm, lv, st = _level(10, 12, 2, precond, lam=5.0)
        args = lambda s: (s["u"], s["v1"], s["v2"], s["u_w"], s["Iu"], s["rho0"], lv["a"],
                          lv["b"], lv["c"], lv["m1"], lv["m2"], lv["M"], prm.lam, prm.alpha0,
                          prm.alpha1)
        E0 = tgv_energy(*args(st))
        for _ in range(25000):
            tgv_iteration(st, lv, prm)
        E = tgv_energy(*args(st))
        assert E < 0.8 * E0
        finals.append(E)
    assert abs(finals[0] - finals[1]) <= 1e-6 * finals[0]


def test_tgv_recovers_a_fronto_parallel_plane():
    # end to end: the full method with the TGV-L1 energy on a rendered plane
    p = synth.fronto_plane(0, model="equidistant", depth=2.0, cycles_per_px=0.05,
                           baseline=0.2, supersample=4)
    prm = oracle.Params(lam=p["lam"], eps=p["eps"], regularizer="tgv")
    r = oracle.solve(p["I0"], p["I1"], p["cam0"], p["cam1"], p["R"], p["t"], p["levels"],
                     p["warps"], p["iters"], prm)
    import scipy.ndimage as nd
    cam = oracle.calib_from_dict(p["cam0"])
    H, W = p["I0"].shape
    py, px = np.mgrid[0:H, 0:W].astype(float)
    ray = oracle.unproject(cam, px, py)
    theta = np.degrees(np.arccos(np.clip(ray[..., 2], -1, 1)))
    sel = nd.binary_erosion(r["mask"], iterations=4) & (theta < 60.0)
    Z = r["depth"] * ray[..., 2]
    rel = Z[sel] / 2.0 - 1.0
    assert abs(np.median(rel)) <= 0.01 and np.median(np.abs(rel)) <= 0.025

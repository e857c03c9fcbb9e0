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


def z_ordered(p):
    """The same map stored along a Z-order curve of the means (the storage
    order the benchmark uses: a view's visible Gaussians form long runs, so
    warps of the per-Gaussian kernels cull together).  The set of Gaussians
    is unchanged."""
    import torch
    from .mapping import morton_order
    perm = morton_order(torch.as_tensor(p["means"], dtype=torch.float64)).numpy()
    out = {k: (v[perm] if isinstance(v, np.ndarray) and k != "sh" else v) for k, v in p.items()}
    out["sh"] = np.ascontiguousarray(p["sh"][:, perm])
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        out[k] = np.ascontiguousarray(out[k])
    return out


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


# --------------------------------------------------------------------------
# Streaming keyframes (drone-like loop through the room).
# --------------------------------------------------------------------------
EUROC_W, EUROC_H, EUROC_F = 752, 480, 460.0


def drone_loop(n_kf, seed=SEED_BASE + 5, length=5.0, width=EUROC_W, height=EUROC_H, f=EUROC_F,
               centre=(0.0, -0.2, 1.6), jitter_m=0.02, jitter_deg=4.0):
    """n_kf grayscale keyframes evenly spaced on a closed horizontal loop of the
    given length (a circle in x-z with a +-0.1 m vertical wave), the camera
    looking along the direction of travel, pitched 10 degrees down, with
    seeded position and orientation jitter.  Returns camera dicts."""
    rng = np.random.default_rng(seed)
    r = length / (2 * np.pi)
    views = []
    for k in range(n_kf):
        th = 2 * np.pi * k / n_kf
        c = np.array([centre[0] + r * np.cos(th), centre[1] + 0.1 * np.sin(3 * th),
                      centre[2] + r * np.sin(th)]) + rng.normal(0, jitter_m, 3)
        fwd = np.array([-np.sin(th), 0.0, np.cos(th)])  # tangent of the loop
        yaw = np.arctan2(fwd[0], fwd[2])
        R_cw = (_rotation_from_axis_angle([0, 1, 0], yaw) @
                _rotation_from_axis_angle([1, 0, 0], np.deg2rad(-10.0)) @
                _rotation_from_axis_angle(rng.normal(size=3), np.deg2rad(rng.uniform(0, jitter_deg))))
        R = R_cw.T
        t = -R @ c
        views.append(camera(width, height, f, f, R=R.astype(np.float32), t=t.astype(np.float32),
                            channels=1))
    return views


def room_textures(seed=SEED_BASE + 5, n_boxes=20):
    """The room's faces (as in room_scene with the same seed) with a seeded
    grayscale texture per face: base + amp * sin(2 pi a/p) sin(2 pi b/p) over
    the face's metric coordinates (a, b)."""
    rng = np.random.default_rng(seed)
    faces = _room_faces(rng, n_boxes)
    tex = [(rng.uniform(0.25, 0.75), rng.uniform(0.1, 0.2), rng.uniform(0.12, 0.45))
           for _ in faces]
    return faces, tex


def ray_cast(view, faces, tex, device="cpu"):
    """Depth (camera z) and grayscale image of the textured room seen from a
    view, by intersecting each pixel's ray (through the integer pixel
    coordinate) with every axis-aligned face; nearest hit wins.  Torch on the
    given device; returns float32 numpy arrays [H][W]."""
    import torch
    H, W = view["height"], view["width"]
    dt = torch.float64
    R = torch.as_tensor(np.asarray(view["R"], np.float64), dtype=dt, device=device)
    t = torch.as_tensor(np.asarray(view["t"], np.float64), dtype=dt, device=device)
    c = -R.T @ t
    ys, xs = torch.meshgrid(torch.arange(H, dtype=dt, device=device),
                            torch.arange(W, dtype=dt, device=device), indexing="ij")
    d_cam = torch.stack([(xs - view["cx"]) / view["fx"], (ys - view["cy"]) / view["fy"],
                         torch.ones_like(xs)], dim=-1)
    d = d_cam @ R  # rows: R^T d_cam
    best = torch.full((H, W), float("inf"), dtype=dt, device=device)
    gray = torch.zeros((H, W), dtype=dt, device=device)
    for (O, U, Vv), (base, amp, per) in zip(faces, tex):
        O, U, Vv = (np.asarray(a, np.float64) for a in (O, U, Vv))
        n_ax = int(np.argmax(np.abs(np.cross(U, Vv))))  # the face's normal axis
        u_ax, v_ax = int(np.argmax(np.abs(U))), int(np.argmax(np.abs(Vv)))
        du = d[..., n_ax]
        s = (O[n_ax] - float(c[n_ax])) / torch.where(du == 0, torch.full_like(du, 1e-30), du)
        a = (c[u_ax] + s * d[..., u_ax] - O[u_ax]) / U[u_ax]
        b = (c[v_ax] + s * d[..., v_ax] - O[v_ax]) / Vv[v_ax]
        hit = (s > 1e-6) & (a >= 0) & (a <= 1) & (b >= 0) & (b <= 1) & (s < best)
        val = base + amp * torch.sin(2 * np.pi * a * abs(U[u_ax]) / per) * \
            torch.sin(2 * np.pi * b * abs(Vv[v_ax]) / per)
        best = torch.where(hit, s, best)
        gray = torch.where(hit, val, gray)
    depth = best  # ray parameter along d with d_cam.z = 1, i.e. camera z
    return depth.float().cpu().numpy(), gray.float().cpu().numpy()


def dso_points(view, depth, gray, n_points, seed, block=4, idepth_sigma=0.01, sh_degree=3,
               opacity=0.1):
    """A semi-dense DSO-like point set turned into new Gaussians: per block x
    block pixel block the pixel of largest central-difference gradient, the
    n_points strongest of those, depth from the ray cast with inverse-depth
    noise N(0, idepth_sigma), back-projected; isotropic scale of one block's
    footprint, identity rotation, the given opacity, SH DC from the pixel's
    gray value (the rest zero)."""
    rng = np.random.default_rng(seed)
    H, W = gray.shape
    gx = np.zeros_like(gray)
    gy = np.zeros_like(gray)
    gx[:, 1:-1] = 0.5 * (gray[:, 2:] - gray[:, :-2])
    gy[1:-1, :] = 0.5 * (gray[2:, :] - gray[:-2, :])
    mag = np.hypot(gx, gy)
    mag[~np.isfinite(depth)] = -1.0
    Hb, Wb = H // block, W // block
    blocks = mag[:Hb * block, :Wb * block].reshape(Hb, block, Wb, block).transpose(0, 2, 1, 3)
    blocks = blocks.reshape(Hb, Wb, block * block)
    arg = blocks.argmax(axis=2)
    val = np.take_along_axis(blocks, arg[..., None], axis=2)[..., 0]
    by, bx = np.meshgrid(np.arange(Hb), np.arange(Wb), indexing="ij")
    py = by * block + arg // block
    px = bx * block + arg % block
    order = np.argsort(-val, axis=None, kind="stable")[:n_points]
    py, px = py.reshape(-1)[order], px.reshape(-1)[order]
    keep = val.reshape(-1)[order] > 0
    py, px = py[keep], px[keep]
    z = depth[py, px].astype(np.float64)
    iz = 1.0 / z + rng.normal(0.0, idepth_sigma, z.shape)
    z = 1.0 / np.clip(iz, 1e-3, None)
    xc = np.stack([(px - view["cx"]) / view["fx"] * z, (py - view["cy"]) / view["fy"] * z, z], 1)
    R = np.asarray(view["R"], np.float64)
    t = np.asarray(view["t"], np.float64)
    xw = (xc - t) @ R  # R^T (x_c - t)
    n = xw.shape[0]
    K = (sh_degree + 1) ** 2
    sh = np.zeros((K, n, 3))
    sh[0] = ((gray[py, px] - 0.5) * 2.0 * np.sqrt(np.pi))[:, None]  # DC of a gray colour
    q = np.zeros((n, 4))
    q[:, 0] = 1.0
    return dict(
        means=np.ascontiguousarray(xw, np.float32),
        log_scales=np.ascontiguousarray(
            np.repeat(np.log(z * 0.5 * block / view["fx"])[:, None], 3, 1), np.float32),
        quats=np.ascontiguousarray(q, np.float32),
        opacity_logits=np.full(n, np.log(opacity / (1 - opacity)), np.float32),
        sh=np.ascontiguousarray(sh, np.float32),
        sh_degree=int(sh_degree),
    )


def streaming_keyframes(n_kf, points_per_kf, seed=SEED_BASE + 5, width=EUROC_W, height=EUROC_H,
                        f=EUROC_F, device="cpu", sh_degree=3):
    """Yields (view, target [1][H][W], new Gaussians) for each keyframe of the
    streaming workload: ray-cast textured room as the keyframe image, its
    DSO-like points as the Gaussians inserted with it."""
    scale = width / EUROC_W
    views = drone_loop(n_kf, seed, width=width, height=height, f=f)
    faces, tex = room_textures(seed)
    for k, v in enumerate(views):
        depth, gray = ray_cast(v, faces, tex, device)
        new = dso_points(v, depth, gray, points_per_kf, seed + 1000 + k,
                         block=max(2, int(round(4 * scale))), sh_degree=sh_degree)
        yield v, gray[None].astype(np.float32), new

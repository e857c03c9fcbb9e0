"""FP64 CPU oracle of the Gaussian-splatting mapping step -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU product path never does, and
the two share no code: the oracle is plain C (``gs_oracle.c``, double
precision, no fused multiply-add contraction) driven through ctypes, plus the
Python composition below.

Each wrapper cites the part of the paper it restates:
  * projection, depth sorting and front-to-back blending -- paper Sec. II
    (Related Work, the 3DGS paragraph) and Sec. III-B (Dense Reconstruction:
    the original differentiable tile-based rasteriser, RGB colour);
  * the photometric loss -- Eq. 2 (read as L1 + lambda (1 - SSIM));
  * the optimiser -- Sec. IV-A (default 3DGS configuration, i.e. Adam).

Every function here is pinned by the ``-m "not gpu"`` tests against closed
forms, brute force, library routines (scipy spherical harmonics) and central
finite differences, not against itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgs_oracle.so")
_lock = threading.Lock()
_lib = None

# Guard bits (mirrors of the #defines in gs_oracle.c, which is the authority).
GUARD_RECT, GUARD_NEAR, GUARD_DET, GUARD_KINK, GUARD_DEPTH, GUARD_TIGHT, GUARD_RADIUS = (
    1, 2, 4, 8, 16, 32, 64)
GPX_ALPHA, GPX_TRANS, GPX_POWER, GPX_KINK = 1, 2, 4, 16

NEAR_Z = 0.2
# Tile rects cut to the tiles that can receive alpha >= 1/255 (reading C19),
# the default of the GPU path too; tight=False gives the plain 3-sigma squares.
TIGHT_RECT = True


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into libgs_oracle.so next to it (gcc, -O2, strict
    FP64, OpenMP for the optional multi-threaded loops)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.oracle_project.restype = ctypes.c_int
            lib.oracle_bin.restype = ctypes.c_int64
            lib.oracle_bin_spans.restype = ctypes.c_int64
            lib.oracle_loss_l1_ssim.restype = ctypes.c_double
            lib.oracle_set_threads(ctypes.c_int(1))
            _lib = lib
    return _lib


def set_threads(k: int) -> None:
    """Host threads of the oracle's parallel loops (default 1; the tests use
    one thread, the benchmark's all-core CPU baseline more)."""
    _L().oracle_set_threads(ctypes.c_int(int(k)))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(v):
    return ctypes.c_int(int(v))


def _f(v):
    return ctypes.c_double(float(v))


def cam_vector(view) -> np.ndarray:
    """R[9] (world->camera), t[3], fx, fy, cx, cy as the C code expects."""
    return _d(np.concatenate([np.asarray(view["R"], np.float64).reshape(9),
                              np.asarray(view["t"], np.float64).reshape(3),
                              [view["fx"], view["fy"], view["cx"], view["cy"]]]))


def tile_grid(width, height, tile_w, tile_h):
    return (width + tile_w - 1) // tile_w, (height + tile_h - 1) // tile_h


# --------------------------------------------------------------------------
# Single steps.
# --------------------------------------------------------------------------
def sh_basis(degree: int, direction) -> np.ndarray:
    out = np.zeros(16)
    _L().oracle_sh_basis(_i(degree), _p(_d(direction)), _p(out))
    return out[: (degree + 1) ** 2]


def ssim_window() -> np.ndarray:
    out = np.zeros((11, 11))
    _L().oracle_ssim_window(_p(out))
    return out


def project(params, view, tile_w=16, tile_h=16, near_z=NEAR_Z, tight=TIGHT_RECT):
    """Projection of all Gaussians into one view (Sec. II / Sec. III-B).
    tight: tile rects cut to the tiles that can receive alpha >= 1/255
    (reading C19 in gs_oracle.c); the rendered image is the same."""
    n = params["means"].shape[0]
    deg = int(params["sh_degree"])
    means, ls, q = _d(params["means"]), _d(params["log_scales"]), _d(params["quats"])
    ol, sh = _d(params["opacity_logits"]), _d(params["sh"])
    out = dict(mean2d=np.zeros((n, 2)), depth=np.zeros(n), cov2d=np.zeros((n, 3)),
               conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
               clamped=np.zeros((n, 3), np.int32), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), tiles_touched=np.zeros(n, np.int32),
               guard=np.zeros(n, np.int32))
    nvis = _L().oracle_project(
        _i(n), _i(deg), _p(means), _p(ls), _p(q), _p(ol), _p(sh), _p(cam_vector(view)),
        _i(view["width"]), _i(view["height"]), _i(tile_w), _i(tile_h), _f(near_z),
        _p(out["mean2d"]), _p(out["depth"]), _p(out["cov2d"]), _p(out["conic"]),
        _p(out["opacity"]), _p(out["rgb"]), _p(out["clamped"]), _p(out["radius"]),
        _p(out["rect"]), _p(out["tiles_touched"]), _p(out["guard"]), _i(1 if tight else 0))
    out["n_visible"] = nvis
    return out


def bin_tiles(depth_key, rect, tiles_touched, tiles_x, tiles_y, spans_of=None, tile=(16, 16)):
    """Per-tile Gaussian lists in (FP32 depth, index) order (Sec. II depth sorting).
    Every tile of each rect, or, with spans_of = a projection made with
    tight=True, each rect's row spans (reading C19)."""
    n = len(tiles_touched)
    dk = np.ascontiguousarray(depth_key, dtype=np.float32)
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    tt = np.ascontiguousarray(tiles_touched, dtype=np.int32)
    total = int(tt.astype(np.int64).sum())
    start = np.zeros(tiles_x * tiles_y + 1, np.int64)
    lst = np.zeros(max(total, 1), np.int32)
    if spans_of is None:
        got = _L().oracle_bin(_i(n), _p(dk), _p(rect), _p(tt), _i(tiles_x), _i(tiles_y),
                              _p(start), _p(lst), ctypes.c_int64(lst.size))
    else:
        got = _L().oracle_bin_spans(
            _i(n), _p(dk), _p(rect), _p(tt), _p(_d(spans_of["mean2d"])),
            _p(_d(spans_of["cov2d"])), _p(_d(spans_of["opacity"])), _i(tile[0]), _i(tile[1]),
            _i(tiles_x), _i(tiles_y), _p(start), _p(lst), ctypes.c_int64(lst.size))
    assert got == total
    return start, lst[:total]


def render(proj, tile_start, tile_list, view, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0)):
    """Front-to-back compositing of one view from tile lists (Sec. II, Sec. III-B).
    guard_px: per pixel, the guard bits (GPX_*) of the decisions taken there
    whose FP64 margin FP32 may not resolve; guard_g: per Gaussian, the same
    bits of its own decisions at any pixel (its alpha next to 1/255 or to
    the 0.99 clamp, its power next to 0, T(1 - alpha) next to 1e-4 where it
    is the Gaussian that would end the pixel)."""
    W, H, C = int(view["width"]), int(view["height"]), int(view.get("channels", 3))
    n = proj["mean2d"].shape[0]
    out = dict(image=np.zeros((C, H, W)), final_T=np.zeros((H, W)),
               last_idx=np.zeros((H, W), np.int32), n_eval=np.zeros((H, W), np.int32),
               n_included=np.zeros((H, W), np.int32), guard_px=np.zeros((H, W), np.int32),
               guard_g=np.zeros(n, np.int32))
    _L().oracle_render(
        _i(n), _p(_d(proj["mean2d"])), _p(_d(proj["conic"])), _p(_d(proj["opacity"])),
        _p(_d(proj["rgb"])), _p(np.ascontiguousarray(tile_start, np.int64)),
        _p(np.ascontiguousarray(tile_list, np.int32)), _i(W), _i(H), _i(tile_w), _i(tile_h),
        _i(C), _p(_d(bg)), _p(out["image"]), _p(out["final_T"]), _p(out["last_idx"]),
        _p(out["n_eval"]), _p(out["n_included"]), _p(out["guard_px"]), _p(out["guard_g"]))
    return out


def render_brute(proj, view, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0), use_rect=True):
    """Per-pixel brute force over all Gaussians in (depth, index) order."""
    W, H, C = int(view["width"]), int(view["height"]), int(view.get("channels", 3))
    n = proj["mean2d"].shape[0]
    out = dict(image=np.zeros((C, H, W)), final_T=np.zeros((H, W)),
               n_included=np.zeros((H, W), np.int32))
    rect = np.ascontiguousarray(proj["rect"], np.int32)
    _L().oracle_render_brute(
        _i(n), _p(_d(proj["mean2d"])), _p(_d(proj["conic"])), _p(_d(proj["opacity"])),
        _p(_d(proj["rgb"])), _p(np.ascontiguousarray(proj["depth"], np.float32)),
        _p(np.ascontiguousarray(proj["tiles_touched"], np.int32)),
        _p(rect) if use_rect else None, _i(W), _i(H), _i(tile_w), _i(tile_h), _i(C),
        _p(_d(bg)), _p(out["image"]), _p(out["final_T"]), _p(out["n_included"]))
    return out


def render_bwd(proj, tile_start, tile_list, view, dL_dimg, tile_w=16, tile_h=16,
               bg=(0.0, 0.0, 0.0)):
    """Adjoint of `render`: screen-space gradients per Gaussian, and the
    homodirectional mean gradient dmean2d_abs (per-pixel contributions summed
    by absolute value per component; the AbsGS density-control statistic)."""
    W, H, C = int(view["width"]), int(view["height"]), int(view.get("channels", 3))
    n = proj["mean2d"].shape[0]
    g = dict(dmean2d=np.zeros((n, 2)), dconic=np.zeros((n, 3)), dopacity=np.zeros(n),
             drgb=np.zeros((n, 3)), dmean2d_abs=np.zeros((n, 2)))
    _L().oracle_render_bwd(
        _i(n), _p(_d(proj["mean2d"])), _p(_d(proj["conic"])), _p(_d(proj["opacity"])),
        _p(_d(proj["rgb"])), _p(np.ascontiguousarray(tile_start, np.int64)),
        _p(np.ascontiguousarray(tile_list, np.int32)), _i(W), _i(H), _i(tile_w), _i(tile_h),
        _i(C), _p(_d(bg)), _p(_d(np.asarray(dL_dimg).reshape(C, H, W))),
        _p(g["dmean2d"]), _p(g["dconic"]), _p(g["dopacity"]), _p(g["drgb"]),
        _p(g["dmean2d_abs"]))
    return g


def zero_grads(params):
    n = params["means"].shape[0]
    K = (int(params["sh_degree"]) + 1) ** 2
    return dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                opacity_logits=np.zeros(n), sh=np.zeros((K, n, 3)))


def project_bwd(params, view, g2d, grads=None, tile_w=16, tile_h=16, near_z=NEAR_Z,
                tight=TIGHT_RECT):
    """Adjoint of `project`: parameter gradients, accumulated into `grads`."""
    if grads is None:
        grads = zero_grads(params)
    n = params["means"].shape[0]
    _L().oracle_project_bwd(
        _i(n), _i(int(params["sh_degree"])), _p(_d(params["means"])),
        _p(_d(params["log_scales"])), _p(_d(params["quats"])),
        _p(_d(params["opacity_logits"])), _p(_d(params["sh"])), _p(cam_vector(view)),
        _i(view["width"]), _i(view["height"]), _i(tile_w), _i(tile_h), _f(near_z),
        _p(_d(g2d["dmean2d"])), _p(_d(g2d["dconic"])), _p(_d(g2d["dopacity"])),
        _p(_d(g2d["drgb"])), _p(grads["means"]), _p(grads["log_scales"]), _p(grads["quats"]),
        _p(grads["opacity_logits"]), _p(grads["sh"]), _i(1 if tight else 0))
    return grads


def loss_l1_ssim(image, target, lam, want_grad=True, want_map=False):
    """Eq. 2 as L = (1-lam) mean|I-I_gt| + lam (1 - mean SSIM); returns (L, dL/dI[, map])."""
    img, tgt = _d(image), _d(target)
    if img.ndim == 2:
        img, tgt = img[None], tgt[None]
    C, H, W = img.shape
    d = np.zeros_like(img) if want_grad else None
    smap = np.zeros_like(img) if want_map else None
    L = _L().oracle_loss_l1_ssim(_p(img), _p(tgt), _i(C), _i(H), _i(W), _f(lam),
                                 _p(d) if d is not None else None,
                                 _p(smap) if smap is not None else None)
    if want_map:
        return L, d, smap
    return L, d


def adam(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step in place on float64 arrays (Sec. IV-A default optimiser)."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    gg = _d(g)
    _L().oracle_adam(ctypes.c_int64(p.size), _p(p), _p(gg), _p(m), _p(v), _f(lr), _f(b1),
                     _f(b2), _f(eps), _i(step))


def adam_masked(p, g, m, v, lr, step, mask, b1=0.9, b2=0.999, eps=1e-15):
    """The visibility-masked variant of the Adam step (no counterpart in the
    paper, whose optimiser is dense): `adam` on the elements where mask is
    true, the others left untouched (in place)."""
    idx = np.flatnonzero(np.asarray(mask).reshape(-1))
    pp, mm, vv = (np.ascontiguousarray(a.reshape(-1)[idx]) for a in (p, m, v))
    adam(pp, np.asarray(g, np.float64).reshape(-1)[idx], mm, vv, lr, step, b1, b2, eps)
    for a, b in ((p, pp), (m, mm), (v, vv)):
        a.reshape(-1)[idx] = b


# --------------------------------------------------------------------------
# Composition: a whole view, a whole mapping iteration.
# --------------------------------------------------------------------------
def forward_view(params, view, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0), near_z=NEAR_Z,
                 tight=TIGHT_RECT):
    """project -> bin -> render for one view; returns (proj, tile_start, list, render_out)."""
    proj = project(params, view, tile_w, tile_h, near_z, tight)
    tx, ty = tile_grid(view["width"], view["height"], tile_w, tile_h)
    start, lst = bin_tiles(proj["depth"].astype(np.float32), proj["rect"],
                           proj["tiles_touched"], tx, ty, proj if tight else None,
                           (tile_w, tile_h))
    out = render(proj, start, lst, view, tile_w, tile_h, bg)
    return proj, start, lst, out


PARAM_GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def iteration(params, views, targets, lam, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0),
              near_z=NEAR_Z, stats=None, tight=TIGHT_RECT):
    """Loss (mean over views) and parameter gradients (sum of per-view adjoints).
    With stats = (accum, denom) the density-control statistic of this
    iteration is added to them (densify_stats)."""
    grads = zero_grads(params)
    total = 0.0
    renders = []
    V = len(views)
    for view, tgt in zip(views, targets):
        proj, start, lst, out = forward_view(params, view, tile_w, tile_h, bg, near_z, tight)
        L, dimg = loss_l1_ssim(out["image"], tgt, lam)
        total += L / V
        g2d = render_bwd(proj, start, lst, view, dimg / V, tile_w, tile_h, bg)
        project_bwd(params, view, g2d, grads, tile_w, tile_h, near_z, tight)
        if stats is not None:
            densify_stats(stats[0], stats[1], view, proj["tiles_touched"], g2d["dmean2d_abs"])
        renders.append(out)
    return total, grads, renders


# --------------------------------------------------------------------------
# Adaptive density control (paper Sec. III-B): every so many iterations,
# Gaussians with a high homodirectional view-space position gradient (the
# AbsGS criterion) are cloned when small and split when large, and Gaussians
# of low opacity are pruned; splitting and cloning use the original 3DGS
# parameters.  Readings: the statistic is the gradient with respect to the
# projected mean in normalised device coordinates (x_ndc = 2 x_px / W - 1,
# so d/dx_ndc = W/2 d/dx_px), its per-pixel contributions summed by absolute
# value per component, the Euclidean norm of that pair added once per
# (iteration, view) in which the Gaussian touches a tile, and averaged over
# those counts.
# --------------------------------------------------------------------------
DENSIFY_DEFAULTS = dict(grad_threshold=0.0004, percent_dense=0.01, min_opacity=0.005,
                        split_shrink=1.6)

# categories of densify_categories
PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3


def densify_stats(accum, denom, view, touched, dmean2d_abs):
    """Add one view's homodirectional statistic: for every Gaussian touching a
    tile, accum += |(W/2 sum|dL/dx|, H/2 sum|dL/dy|)|, denom += 1 (in place)."""
    vis = np.asarray(touched) > 0
    hx = np.asarray(dmean2d_abs, np.float64)[:, 0] * (0.5 * view["width"])
    hy = np.asarray(dmean2d_abs, np.float64)[:, 1] * (0.5 * view["height"])
    accum[vis] += np.hypot(hx, hy)[vis]
    denom[vis] += 1.0


def densify_categories(params, accum, denom, extent, cfg=None):
    """Per Gaussian: PRUNE if its opacity is below min_opacity (first); else
    CLONE if its mean statistic reaches grad_threshold and its largest scale
    is at most percent_dense * extent; SPLIT if the statistic reaches the
    threshold and the Gaussian is larger; KEEP otherwise."""
    c = dict(DENSIFY_DEFAULTS, **(cfg or {}))
    ol = np.asarray(params["opacity_logits"], np.float64)
    opacity = 1.0 / (1.0 + np.exp(-ol))
    smax = np.exp(np.max(np.asarray(params["log_scales"], np.float64), axis=1))
    accum = np.asarray(accum, np.float64)
    denom = np.asarray(denom, np.float64)
    stat = np.where(denom > 0, accum / np.where(denom > 0, denom, 1.0), 0.0)
    high = (denom > 0) & (stat >= c["grad_threshold"])
    small = smax <= c["percent_dense"] * extent
    cat = np.full(ol.shape[0], KEEP, np.int32)
    cat[high & small] = CLONE
    cat[high & ~small] = SPLIT
    cat[opacity < c["min_opacity"]] = PRUNE
    return cat


def densify_apply(params, moments, cat, samples, cfg=None):
    """The map after density control, in this order: the kept Gaussians (KEEP
    and the originals of CLONE) by index, then the clones by index, then two
    children per SPLIT Gaussian by index.  A clone copies its original. A
    child c of Gaussian i has mean mu_i + R(q_i / |q_i|) (s_i * samples[i, c])
    (samples: standard normal draws, passed in), log-scales reduced by
    log(split_shrink), and the rotation, opacity and SH of its parent.
    moments: dict name -> (m, v) per group in the params layout; kept
    Gaussians keep theirs, new ones start at zero."""
    from scipy.spatial.transform import Rotation
    c = dict(DENSIFY_DEFAULTS, **(cfg or {}))
    cat = np.asarray(cat)
    keep = (cat == KEEP) | (cat == CLONE)
    clone = cat == CLONE
    split = np.flatnonzero(cat == SPLIT)
    mu = np.asarray(params["means"], np.float64)
    ls = np.asarray(params["log_scales"], np.float64)
    q = np.asarray(params["quats"], np.float64)
    samples = np.asarray(samples, np.float64).reshape(-1, 2, 3)
    out = {}
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        a = np.asarray(params[k], np.float64)
        out[k] = np.concatenate([a[keep], a[clone], np.repeat(a[split], 2, axis=0)])
    sh = np.asarray(params["sh"], np.float64)
    out["sh"] = np.concatenate([sh[:, keep], sh[:, clone], np.repeat(sh[:, split], 2, axis=1)],
                               axis=1)
    if split.size:
        Rm = Rotation.from_quat(q[split], scalar_first=True).as_matrix()  # normalises
        s = np.exp(ls[split])
        child = mu[split][:, None, :] + np.einsum("nij,ncj->nci", Rm, s[:, None, :] *
                                                  samples[split])
        base = keep.sum() + clone.sum()
        out["means"][base:] = child.reshape(-1, 3)
        out["log_scales"][base:] -= np.log(c["split_shrink"])
    out["sh_degree"] = params["sh_degree"]
    new_moments = {}
    n_new = clone.sum() + 2 * split.size
    for k, (m, v) in (moments or {}).items():
        m, v = np.asarray(m, np.float64), np.asarray(v, np.float64)
        if k == "sh":
            z = np.zeros((m.shape[0], n_new, m.shape[2]))
            new_moments[k] = (np.concatenate([m[:, keep], z], 1), np.concatenate([v[:, keep], z], 1))
        else:
            z = np.zeros((n_new,) + m.shape[1:])
            new_moments[k] = (np.concatenate([m[keep], z]), np.concatenate([v[keep], z]))
    return out, new_moments


# --------------------------------------------------------------------------
# Gaussian-pyramid targets (paper Sec. III-B: the keyframe image is smoothed
# and down-sampled repeatedly; training starts on the coarsest level and moves
# to finer ones).  Readings: the 5-tap binomial kernel [1, 4, 6, 4, 1] / 16
# applied along each axis, borders mirrored without repeating the edge pixel
# (d c b | a b c d | c b a), then every second pixel kept starting at 0, so
# level L+1 has ceil(W/2) x ceil(H/2) pixels and its pixel i sits on pixel
# 2i of level L (intrinsics fx/2, fy/2, cx/2, cy/2).
# --------------------------------------------------------------------------
PYR_KERNEL = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def pyr_down(img):
    """One pyramid level of a [C][H][W] image (float64)."""
    from scipy.ndimage import convolve1d
    a = np.asarray(img, np.float64)
    a = convolve1d(a, PYR_KERNEL, axis=-1, mode="mirror")
    a = convolve1d(a, PYR_KERNEL, axis=-2, mode="mirror")
    return a[..., ::2, ::2]


def pyr_view(view):
    """The camera of the next pyramid level."""
    return dict(view, width=(view["width"] + 1) // 2, height=(view["height"] + 1) // 2,
                fx=view["fx"] / 2, fy=view["fy"] / 2, cx=view["cx"] / 2, cy=view["cy"] / 2)


# --------------------------------------------------------------------------
# Point-cloud densification (paper Sec. III-A).  Pixel selection: per block
# the pixel of largest image gradient, if above the pass threshold, repeated
# on larger blocks with lower thresholds where nothing was selected yet.
# Readings: central-difference gradient (zero on the one-pixel border),
# compared as the squared magnitude; pass k uses blocks of block * 2^k pixels
# (partial blocks at the right and bottom edges included) and the squared
# threshold thr_sq[k]; ties go to the first pixel in raster order; a pass-k
# block is skipped if any of its pixels was selected in an earlier pass.
# Interpolation: on the pixels of a grid of step `grid` whose squared
# gradient is below flat_sq and that were not selected, the depth is the mean
# of the vertex depths of the first (lowest-index) triangle containing the
# pixel (closed triangles), none outside the triangulation.
# --------------------------------------------------------------------------
def grad_sq(gray):
    g = np.asarray(gray, np.float64)
    gx = np.zeros_like(g)
    gy = np.zeros_like(g)
    gx[1:-1, 1:-1] = 0.5 * (g[1:-1, 2:] - g[1:-1, :-2])
    gy[1:-1, 1:-1] = 0.5 * (g[2:, 1:-1] - g[:-2, 1:-1])
    return gx * gx + gy * gy


def select_pixels(gray, block, thr_sq):
    """int32 [H][W]: 0, or k + 1 for a pixel selected in pass k."""
    g2 = grad_sq(gray)
    H, W = g2.shape
    sel = np.zeros((H, W), np.int32)
    for k, t in enumerate(thr_sq):
        s = block << k
        for y0 in range(0, H, s):
            for x0 in range(0, W, s):
                if np.any(sel[y0:y0 + s, x0:x0 + s]):
                    continue
                reg = g2[y0:y0 + s, x0:x0 + s]
                i = int(np.argmax(reg))  # first maximum in raster order
                if reg.flat[i] >= t:
                    sel[y0 + i // reg.shape[1], x0 + i % reg.shape[1]] = k + 1
    return sel


def interp_depth(tri, xy, depth, gray, selected, grid, flat_sq):
    """float64 [ceil(H/grid)][ceil(W/grid)] depths (0 where no point)."""
    g2 = grad_sq(gray)
    H, W = g2.shape
    out = np.zeros(((H + grid - 1) // grid, (W + grid - 1) // grid))
    P = np.asarray(xy, np.int64)
    T = np.asarray(tri, np.int64)
    for gy in range(out.shape[0]):
        for gx in range(out.shape[1]):
            x, y = gx * grid, gy * grid
            if selected[y, x] or not g2[y, x] < flat_sq:
                continue
            for t, (a, b, c) in enumerate(T):
                e = [(P[v][0] - P[u][0]) * (y - P[u][1]) - (P[v][1] - P[u][1]) * (x - P[u][0])
                     for u, v in ((a, b), (b, c), (c, a))]
                if min(e) >= 0:
                    out[gy, gx] = (depth[a] + depth[b] + depth[c]) / 3.0
                    break
    return out

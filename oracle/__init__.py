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
GUARD_RECT, GUARD_NEAR, GUARD_DET, GUARD_KINK, GUARD_DEPTH = 1, 2, 4, 8, 16
GPX_ALPHA, GPX_TRANS, GPX_POWER, GPX_KINK = 1, 2, 4, 16

NEAR_Z = 0.2


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into libgs_oracle.so next to it (gcc, -O2, strict FP64)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
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
            lib.oracle_loss_l1_ssim.restype = ctypes.c_double
            _lib = lib
    return _lib


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


def project(params, view, tile_w=16, tile_h=16, near_z=NEAR_Z):
    """Projection of all Gaussians into one view (Sec. II / Sec. III-B)."""
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
        _p(out["rect"]), _p(out["tiles_touched"]), _p(out["guard"]))
    out["n_visible"] = nvis
    return out


def bin_tiles(depth_key, rect, tiles_touched, tiles_x, tiles_y):
    """Per-tile Gaussian lists in (FP32 depth, index) order (Sec. II depth sorting)."""
    n = len(tiles_touched)
    dk = np.ascontiguousarray(depth_key, dtype=np.float32)
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    tt = np.ascontiguousarray(tiles_touched, dtype=np.int32)
    total = int(tt.astype(np.int64).sum())
    start = np.zeros(tiles_x * tiles_y + 1, np.int64)
    lst = np.zeros(max(total, 1), np.int32)
    got = _L().oracle_bin(_i(n), _p(dk), _p(rect), _p(tt), _i(tiles_x), _i(tiles_y),
                          _p(start), _p(lst), ctypes.c_int64(lst.size))
    assert got == total
    return start, lst[:total]


def render(proj, tile_start, tile_list, view, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0)):
    """Front-to-back compositing of one view from tile lists (Sec. II, Sec. III-B)."""
    W, H, C = int(view["width"]), int(view["height"]), int(view.get("channels", 3))
    n = proj["mean2d"].shape[0]
    out = dict(image=np.zeros((C, H, W)), final_T=np.zeros((H, W)),
               last_idx=np.zeros((H, W), np.int32), n_eval=np.zeros((H, W), np.int32),
               n_included=np.zeros((H, W), np.int32), guard_px=np.zeros((H, W), np.int32))
    _L().oracle_render(
        _i(n), _p(_d(proj["mean2d"])), _p(_d(proj["conic"])), _p(_d(proj["opacity"])),
        _p(_d(proj["rgb"])), _p(np.ascontiguousarray(tile_start, np.int64)),
        _p(np.ascontiguousarray(tile_list, np.int32)), _i(W), _i(H), _i(tile_w), _i(tile_h),
        _i(C), _p(_d(bg)), _p(out["image"]), _p(out["final_T"]), _p(out["last_idx"]),
        _p(out["n_eval"]), _p(out["n_included"]), _p(out["guard_px"]))
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
    """Adjoint of `render`: screen-space gradients per Gaussian."""
    W, H, C = int(view["width"]), int(view["height"]), int(view.get("channels", 3))
    n = proj["mean2d"].shape[0]
    g = dict(dmean2d=np.zeros((n, 2)), dconic=np.zeros((n, 3)), dopacity=np.zeros(n),
             drgb=np.zeros((n, 3)))
    _L().oracle_render_bwd(
        _i(n), _p(_d(proj["mean2d"])), _p(_d(proj["conic"])), _p(_d(proj["opacity"])),
        _p(_d(proj["rgb"])), _p(np.ascontiguousarray(tile_start, np.int64)),
        _p(np.ascontiguousarray(tile_list, np.int32)), _i(W), _i(H), _i(tile_w), _i(tile_h),
        _i(C), _p(_d(bg)), _p(_d(np.asarray(dL_dimg).reshape(C, H, W))),
        _p(g["dmean2d"]), _p(g["dconic"]), _p(g["dopacity"]), _p(g["drgb"]))
    return g


def zero_grads(params):
    n = params["means"].shape[0]
    K = (int(params["sh_degree"]) + 1) ** 2
    return dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                opacity_logits=np.zeros(n), sh=np.zeros((K, n, 3)))


def project_bwd(params, view, g2d, grads=None, tile_w=16, tile_h=16, near_z=NEAR_Z):
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
        _p(grads["opacity_logits"]), _p(grads["sh"]))
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


# --------------------------------------------------------------------------
# Composition: a whole view, a whole mapping iteration.
# --------------------------------------------------------------------------
def forward_view(params, view, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0), near_z=NEAR_Z):
    """project -> bin -> render for one view; returns (proj, tile_start, list, render_out)."""
    proj = project(params, view, tile_w, tile_h, near_z)
    tx, ty = tile_grid(view["width"], view["height"], tile_w, tile_h)
    start, lst = bin_tiles(proj["depth"].astype(np.float32), proj["rect"],
                           proj["tiles_touched"], tx, ty)
    out = render(proj, start, lst, view, tile_w, tile_h, bg)
    return proj, start, lst, out


PARAM_GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def iteration(params, views, targets, lam, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0),
              near_z=NEAR_Z):
    """Loss (mean over views) and parameter gradients (sum of per-view adjoints)."""
    grads = zero_grads(params)
    total = 0.0
    renders = []
    V = len(views)
    for view, tgt in zip(views, targets):
        proj, start, lst, out = forward_view(params, view, tile_w, tile_h, bg, near_z)
        L, dimg = loss_l1_ssim(out["image"], tgt, lam)
        total += L / V
        g2d = render_bwd(proj, start, lst, view, dimg / V, tile_w, tile_h, bg)
        project_bwd(params, view, g2d, grads, tile_w, tile_h, near_z)
        renders.append(out)
    return total, grads, renders

"""ctypes binding of libgs_gb300.so: the C-ABI of include/gs.h, same names.

Argument marshalling only -- every step of the mapping path runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gs.h")

c_int32, c_int64, c_float, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                   ctypes.c_void_p, ctypes.c_size_t)

GS_OK, GS_ERR_INVALID, GS_ERR_CUDA, GS_ERR_CAPACITY, GS_ERR_UNSUPPORTED, GS_ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5
GS_DEV_CAPACITY, GS_DEV_NONFINITE, GS_DEV_SPAN_POOL = 1, 2, 4
GS_MAX_VIEWS, GS_MAX_GROUPS, GS_PLAN_WORDS = 64, 8, 1536
(GS_BUF_COUNTERS, GS_BUF_PROJ, GS_BUF_RECT, GS_BUF_TOUCHED, GS_BUF_RADIUS, GS_BUF_DEPTH_ORDER,
 GS_BUF_TILE_KEYS, GS_BUF_TILE_VALUES, GS_BUF_RANGES, GS_BUF_GRAD2D, GS_BUF_ABSGRAD) = range(11)


class gs_view(ctypes.Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float), ("width", c_int32), ("height", c_int32),
                ("channels", c_int32), ("reserved", c_int32)]


class gs_map(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p),
                ("opacity_logits", c_void_p), ("sh", c_void_p), ("n", c_int32),
                ("sh_degree", c_int32)]


class gs_map_grad(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p),
                ("opacity_logits", c_void_p), ("sh", c_void_p)]


class gs_config(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("smem_batch", c_int32),
                ("pixels_per_thread", c_int32), ("smem_batch_bwd", c_int32),
                ("pixels_per_thread_bwd", c_int32), ("near_z", c_float), ("bg", c_float * 3),
                ("density_stats", c_int32), ("deterministic", c_int32),
                ("tight_rect", c_int32), ("recompute", c_int32)]


class gs_densify_config(ctypes.Structure):
    _fields_ = [("grad_threshold", c_float), ("percent_dense", c_float),
                ("min_opacity", c_float), ("split_shrink", c_float), ("extent", c_float),
                ("reserved", c_int32 * 3)]


class gs_plan(ctypes.Structure):
    _fields_ = [("words", ctypes.c_uint64 * GS_PLAN_WORDS)]


class gs_counters(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("n_instances", ctypes.c_uint32),
                ("n_instances_raw", ctypes.c_uint64), ("loss", c_float),
                ("reserved", ctypes.c_uint32 * 3)]


_P = ctypes.POINTER
_SIGNATURES = {
    "gs_plan_init": (c_int32, [_P(gs_plan), _P(gs_config), c_int32, _P(gs_view), c_int32,
                               c_int64]),
    "gs_plan_workspace_bytes": (c_size_t, [_P(gs_plan)]),
    "gs_plan_view_pass": (c_int32, [_P(gs_plan), c_int32, _P(gs_plan)]),
    "gs_plan_passes": (c_int32, [_P(gs_plan)]),
    "gs_plan_view": (c_int32, [_P(gs_plan), c_int32, _P(c_int64), _P(c_int64), _P(c_int32),
                               _P(c_int32), _P(c_int32)]),
    "gs_plan_totals": (c_int32, [_P(gs_plan), _P(c_int64), _P(c_int64), _P(c_int32)]),
    "gs_plan_buffer": (c_int32, [_P(gs_plan), c_int32, _P(c_size_t), _P(c_size_t)]),
    "gs_project": (c_int32, [_P(gs_plan), _P(gs_map), c_void_p, c_void_p, c_void_p]),
    "gs_bin_sort": (c_int32, [_P(gs_plan), c_int32, c_void_p, c_void_p]),
    "gs_render_fwd": (c_int32, [_P(gs_plan), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_loss_l1_ssim": (c_int32, [_P(gs_plan), c_void_p, c_void_p, c_float, c_float, c_void_p,
                                  c_void_p, c_void_p, c_void_p]),
    "gs_render_bwd": (c_int32, [_P(gs_plan), _P(gs_map), c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, _P(gs_map_grad), c_int32, c_void_p]),
    "gs_loss_l1_ssim_noalloc": (c_int32, [_P(gs_plan), c_void_p, c_void_p, c_float, c_float,
                                          c_void_p, c_void_p, c_void_p]),
    "gs_render_bwd_pixels": (c_int32, [_P(gs_plan), c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p]),
    "gs_project_bwd": (c_int32, [_P(gs_plan), _P(gs_map), c_void_p, c_void_p, _P(gs_map_grad),
                                 c_int32, c_void_p]),
    "gs_project_bwd_adam": (c_int32, [_P(gs_plan), _P(gs_map), c_void_p, c_void_p,
                                      _P(gs_map_grad), _P(gs_map_grad), _P(gs_map_grad),
                                      _P(gs_map_grad), _P(gs_map_grad), _P(c_float), c_float,
                                      c_float, c_float, c_void_p, c_void_p]),
    "gs_adam_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32,
                               _P(c_int64), _P(c_float), c_float, c_float, c_float, c_void_p,
                               c_void_p]),
    "gs_visibility": (c_int32, [_P(gs_plan), c_int32, c_void_p, c_void_p, c_void_p]),
    "gs_adam_step_sparse": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32,
                                      _P(c_int64), _P(c_float), _P(c_int32), c_int32, c_void_p,
                                      c_float, c_float, c_float, c_void_p, c_void_p]),
    "gs_project_bwd_groups": (c_int32, [_P(gs_plan), _P(gs_map), c_void_p, c_void_p,
                                        _P(gs_map_grad), c_void_p, c_void_p]),
    "gs_adam_step_groups": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32,
                                      _P(c_int64), _P(c_float), _P(c_int32), c_int32, c_void_p,
                                      c_float, c_float, c_float, c_void_p, c_void_p]),
    "gs_densify_stats": (c_int32, [_P(gs_plan), c_int32, c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "gs_densify_scratch_bytes": (c_size_t, [c_int32]),
    "gs_densify_count": (c_int32, [_P(gs_map), c_void_p, c_void_p, _P(gs_densify_config),
                                   c_void_p, c_void_p, c_void_p]),
    "gs_densify_apply": (c_int32, [_P(gs_map), _P(gs_map_grad), _P(gs_map_grad), c_void_p,
                                   c_void_p, c_void_p, _P(gs_densify_config), c_void_p, c_int32,
                                   _P(gs_map_grad), _P(gs_map_grad), _P(gs_map_grad), c_void_p,
                                   c_void_p]),
    "gs_pyr_down": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "gs_delaunay": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, _P(c_int32)]),
    "gs_select_pixels": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, _P(c_float),
                                   c_void_p, c_void_p, c_void_p]),
    "gs_interp_depth": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_int32, c_int32, c_int32, c_float, c_void_p, c_void_p,
                                  c_void_p]),
    "gs_read_counters": (c_int32, [_P(gs_plan), c_void_p, _P(gs_counters), c_void_p]),
    "gs_status_string": (ctypes.c_char_p, [c_int32]),
}

_lib = None


class GSError(RuntimeError):
    pass


def header_functions():
    """Names of the functions include/gs.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


def lib():
    """The loaded library (built in place by paper_2409_13055_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GSError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2409_13055_gb300.build` (there is no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, what=""):
    if status != GS_OK:
        msg = lib().gs_status_string(status).decode()
        raise GSError(f"{what}: {msg}" if what else msg)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# --------------------------------------------------------------------------
# Thin wrappers with the C names: tensors in, status checked.
# --------------------------------------------------------------------------
def gs_plan_init(cfg: gs_config, views_host, n_capacity: int, instance_capacity: int) -> gs_plan:
    arr = (gs_view * len(views_host))(*views_host)
    plan = gs_plan()
    check(lib().gs_plan_init(ctypes.byref(plan), ctypes.byref(cfg), len(views_host), arr,
                             int(n_capacity), int(instance_capacity)), "gs_plan_init")
    return plan


def gs_plan_workspace_bytes(plan) -> int:
    return int(lib().gs_plan_workspace_bytes(ctypes.byref(plan)))


def gs_plan_passes(plan) -> int:
    return int(lib().gs_plan_passes(ctypes.byref(plan)))


def gs_plan_view_pass(plan, k) -> gs_plan:
    """The plan of pass k of a recompute plan."""
    out = gs_plan()
    check(lib().gs_plan_view_pass(ctypes.byref(plan), int(k), ctypes.byref(out)),
          "gs_plan_view_pass")
    return out


def gs_plan_view(plan, v):
    vo, po = c_int64(), c_int64()
    to, tx, ty = c_int32(), c_int32(), c_int32()
    check(lib().gs_plan_view(ctypes.byref(plan), int(v), ctypes.byref(vo), ctypes.byref(po),
                             ctypes.byref(to), ctypes.byref(tx), ctypes.byref(ty)), "gs_plan_view")
    return dict(value_offset=vo.value, pixel_offset=po.value, tile_offset=to.value,
                tiles_x=tx.value, tiles_y=ty.value)


def gs_plan_totals(plan):
    tv, tp, tt = c_int64(), c_int64(), c_int32()
    check(lib().gs_plan_totals(ctypes.byref(plan), ctypes.byref(tv), ctypes.byref(tp),
                               ctypes.byref(tt)), "gs_plan_totals")
    return dict(total_values=tv.value, total_pixels=tp.value, total_tiles=tt.value)


def gs_plan_buffer(plan, buf_id):
    o, b = c_size_t(), c_size_t()
    check(lib().gs_plan_buffer(ctypes.byref(plan), int(buf_id), ctypes.byref(o), ctypes.byref(b)),
          "gs_plan_buffer")
    return o.value, b.value


def gs_project(plan, gmap: gs_map, views_dev, ws, stream=None):
    check(lib().gs_project(ctypes.byref(plan), ctypes.byref(gmap), _ptr(views_dev), _ptr(ws),
                           _stream(stream)), "gs_project")


def gs_bin_sort(plan, n, ws, stream=None):
    check(lib().gs_bin_sort(ctypes.byref(plan), int(n), _ptr(ws), _stream(stream)), "gs_bin_sort")


def gs_render_fwd(plan, ws, images, final_T, last_idx, stream=None):
    check(lib().gs_render_fwd(ctypes.byref(plan), _ptr(ws), _ptr(images), _ptr(final_T),
                              _ptr(last_idx), _stream(stream)), "gs_render_fwd")


def gs_loss_l1_ssim(plan, images, targets, lam, view_weight, loss_dev, dL_dimages, ws,
                    stream=None):
    check(lib().gs_loss_l1_ssim(ctypes.byref(plan), _ptr(images), _ptr(targets), float(lam),
                                float(view_weight), _ptr(loss_dev), _ptr(dL_dimages), _ptr(ws),
                                _stream(stream)), "gs_loss_l1_ssim")


def gs_render_bwd(plan, gmap: gs_map, views_dev, ws, final_T, last_idx, dL_dimages,
                  grads: gs_map_grad, accumulate=False, stream=None):
    check(lib().gs_render_bwd(ctypes.byref(plan), ctypes.byref(gmap), _ptr(views_dev), _ptr(ws),
                              _ptr(final_T), _ptr(last_idx), _ptr(dL_dimages),
                              ctypes.byref(grads), 1 if accumulate else 0, _stream(stream)),
          "gs_render_bwd")


def gs_loss_l1_ssim_noalloc(plan, images, targets, lam, view_weight, loss_dev, dL_dimages,
                            stream=None):
    """gs_loss_l1_ssim with the library's fixed scratch instead of a workspace;
    returns the raw status so callers can see GS_ERR_CAPACITY."""
    return lib().gs_loss_l1_ssim_noalloc(ctypes.byref(plan), _ptr(images), _ptr(targets),
                                         float(lam), float(view_weight), _ptr(loss_dev),
                                         _ptr(dL_dimages), _stream(stream))


def gs_render_bwd_pixels(plan, ws, final_T, last_idx, dL_dimages, stream=None):
    check(lib().gs_render_bwd_pixels(ctypes.byref(plan), _ptr(ws), _ptr(final_T), _ptr(last_idx),
                                     _ptr(dL_dimages), _stream(stream)), "gs_render_bwd_pixels")


def gs_project_bwd(plan, gmap: gs_map, views_dev, ws, grads: gs_map_grad, accumulate=False,
                   stream=None):
    check(lib().gs_project_bwd(ctypes.byref(plan), ctypes.byref(gmap), _ptr(views_dev), _ptr(ws),
                               ctypes.byref(grads), 1 if accumulate else 0, _stream(stream)),
          "gs_project_bwd")


def gs_project_bwd_adam(plan, gmap: gs_map, views_dev, ws, params: gs_map_grad, m: gs_map_grad,
                        v: gs_map_grad, group_lr, beta1, beta2, eps, step_dev, grads_acc=None,
                        grads_out=None, stream=None):
    lrs = (c_float * 6)(*[float(x) for x in group_lr])
    check(lib().gs_project_bwd_adam(ctypes.byref(plan), ctypes.byref(gmap), _ptr(views_dev),
                                    _ptr(ws), ctypes.byref(params), ctypes.byref(m),
                                    ctypes.byref(v),
                                    ctypes.byref(grads_acc) if grads_acc is not None else None,
                                    ctypes.byref(grads_out) if grads_out is not None else None,
                                    lrs, float(beta1), float(beta2), float(eps), _ptr(step_dev),
                                    _stream(stream)), "gs_project_bwd_adam")


def gs_adam_step(params, grads, m, v, group_offsets, group_lr, beta1, beta2, eps, step_dev,
                 stream=None):
    ng = len(group_lr)
    offs = (c_int64 * (ng + 1))(*[int(x) for x in group_offsets])
    lrs = (c_float * ng)(*[float(x) for x in group_lr])
    check(lib().gs_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(params.numel()), ng,
                             offs, lrs, float(beta1), float(beta2), float(eps), _ptr(step_dev),
                             _stream(stream)), "gs_adam_step")


def gs_visibility(plan, n, ws, vis, stream=None):
    check(lib().gs_visibility(ctypes.byref(plan), int(n), _ptr(ws), _ptr(vis), _stream(stream)),
          "gs_visibility")


def gs_adam_step_sparse(params, grads, m, v, group_offsets, group_lr, group_strides, n_gauss, vis,
                        beta1, beta2, eps, step_dev, stream=None):
    ng = len(group_lr)
    offs = (c_int64 * (ng + 1))(*[int(x) for x in group_offsets])
    lrs = (c_float * ng)(*[float(x) for x in group_lr])
    strides = (c_int32 * ng)(*[int(x) for x in group_strides])
    check(lib().gs_adam_step_sparse(_ptr(params), _ptr(grads), _ptr(m), _ptr(v),
                                    int(params.numel()), ng, offs, lrs, strides, int(n_gauss),
                                    _ptr(vis), float(beta1), float(beta2), float(eps),
                                    _ptr(step_dev), _stream(stream)), "gs_adam_step_sparse")


GS_GRAD_GROUP = 32


def gs_project_bwd_groups(plan, gmap, views_dev, ws, grads, group_vis, stream=None):
    check(lib().gs_project_bwd_groups(ctypes.byref(plan), ctypes.byref(gmap), _ptr(views_dev),
                                      _ptr(ws), ctypes.byref(grads), _ptr(group_vis),
                                      _stream(stream)), "gs_project_bwd_groups")


def gs_adam_step_groups(params, grads, m, v, group_offsets, group_lr, group_strides, n_gauss,
                        group_vis, beta1, beta2, eps, step_dev, stream=None):
    ng = len(group_lr)
    offs = (c_int64 * (ng + 1))(*[int(x) for x in group_offsets])
    lrs = (c_float * ng)(*[float(x) for x in group_lr])
    strides = (c_int32 * ng)(*[int(x) for x in group_strides])
    check(lib().gs_adam_step_groups(_ptr(params), _ptr(grads), _ptr(m), _ptr(v),
                                    int(params.numel()), ng, offs, lrs, strides, int(n_gauss),
                                    _ptr(group_vis), float(beta1), float(beta2), float(eps),
                                    _ptr(step_dev), _stream(stream)), "gs_adam_step_groups")


def gs_densify_stats(plan, n, ws, accum, denom, stream=None):
    check(lib().gs_densify_stats(ctypes.byref(plan), int(n), _ptr(ws), _ptr(accum), _ptr(denom),
                                 _stream(stream)), "gs_densify_stats")


def gs_densify_scratch_bytes(n) -> int:
    return int(lib().gs_densify_scratch_bytes(int(n)))


def gs_densify_count(gmap, accum, denom, cfg, scratch, counts_dev, stream=None):
    check(lib().gs_densify_count(ctypes.byref(gmap), _ptr(accum), _ptr(denom), ctypes.byref(cfg),
                                 _ptr(scratch), _ptr(counts_dev), _stream(stream)),
          "gs_densify_count")


def gs_densify_apply(gmap, src_m, src_v, accum, denom, samples, cfg, scratch, n_out, dst, dst_m,
                     dst_v, counts_dev, stream=None):
    check(lib().gs_densify_apply(ctypes.byref(gmap), ctypes.byref(src_m), ctypes.byref(src_v),
                                 _ptr(accum), _ptr(denom), _ptr(samples), ctypes.byref(cfg),
                                 _ptr(scratch), int(n_out), ctypes.byref(dst), ctypes.byref(dst_m),
                                 ctypes.byref(dst_v), _ptr(counts_dev), _stream(stream)),
          "gs_densify_apply")


def gs_pyr_down(src, channels, height, width, dst, stream=None):
    check(lib().gs_pyr_down(_ptr(src), int(channels), int(height), int(width), _ptr(dst),
                            _stream(stream)), "gs_pyr_down")


def gs_delaunay(xy):
    """Triangles [T][3] (int32, counter-clockwise) of the Delaunay triangulation
    of the integer points xy [n][2] (host numpy)."""
    import numpy as np
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    n = xy.shape[0]
    cap = max(1, 2 * n)
    tri = np.zeros((cap, 3), np.int32)
    cnt = c_int32(0)
    check(lib().gs_delaunay(xy.ctypes.data, n, tri.ctypes.data, cap, ctypes.byref(cnt)),
          "gs_delaunay")
    return tri[: cnt.value].copy()


def gs_select_pixels(gray, block, thresholds_sq, grad_sq, selected, stream=None):
    H, W = gray.shape
    thr = (c_float * len(thresholds_sq))(*[float(t) for t in thresholds_sq])
    check(lib().gs_select_pixels(_ptr(gray), H, W, int(block), len(thresholds_sq), thr,
                                 _ptr(grad_sq), _ptr(selected), _stream(stream)),
          "gs_select_pixels")


def gs_interp_depth(tri, xy, depth, grad_sq, selected, grid, flat_sq, owner, out, stream=None):
    H, W = grad_sq.shape
    check(lib().gs_interp_depth(_ptr(tri), int(tri.shape[0]), _ptr(xy), _ptr(depth),
                                _ptr(grad_sq), _ptr(selected), H, W, int(grid), float(flat_sq),
                                _ptr(owner), _ptr(out), _stream(stream)), "gs_interp_depth")


def gs_read_counters(plan, ws, stream=None) -> gs_counters:
    c = gs_counters()
    check(lib().gs_read_counters(ctypes.byref(plan), _ptr(ws), ctypes.byref(c), _stream(stream)),
          "gs_read_counters")
    return c


def gs_status_string(status) -> str:
    return lib().gs_status_string(int(status)).decode()

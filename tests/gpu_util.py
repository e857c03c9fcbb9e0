"""Helpers shared by the GPU parity tests: read workspace buffers back, build
the oracle-side guard masks, compare tile lists."""
import numpy as np
import torch

import oracle
from paper_2409_13055_gb300 import binding as B
from paper_2409_13055_gb300 import mapping

# decisions that can change a tile list or a radius (all of them) or a pixel
# value (all but the tight-rect edges, which only move tiles where alpha <
# 1/255, and a radius change that leaves the rect as it is)
FWD_GUARDS = (oracle.GUARD_RECT | oracle.GUARD_NEAR | oracle.GUARD_DET | oracle.GUARD_DEPTH |
              oracle.GUARD_TIGHT | oracle.GUARD_RADIUS)
PIXEL_GUARDS = oracle.GUARD_RECT | oracle.GUARD_NEAR | oracle.GUARD_DET | oracle.GUARD_DEPTH


def gpu_projection(rast: mapping.Rasterizer, n: int, v: int = 0):
    """Per-Gaussian projection outputs of view v from the workspace."""
    V = len(rast.views)
    proj = rast.buffer(B.GS_BUF_PROJ, torch.float32)[: V * n * 12].view(V, n, 12)[v]
    proj = proj.cpu().numpy().astype(np.float64)
    rect = rast.buffer(B.GS_BUF_RECT, torch.int16)[: V * n * 4].view(V, n, 4)[v]
    rect = rect.cpu().numpy().astype(np.int64) & 0xFFFF
    touched = rast.buffer(B.GS_BUF_TOUCHED, torch.int32)[: V * n].view(V, n)[v].cpu().numpy()
    radius = rast.buffer(B.GS_BUF_RADIUS, torch.int32)[: V * n].view(V, n)[v].cpu().numpy()
    depth32 = rast.buffer(B.GS_BUF_PROJ, torch.float32)[: V * n * 12].view(V, n, 12)[v, :, 11]
    return dict(mean2d=proj[:, 0:2] + proj[:, 2:4], conic=proj[:, 4:7], opacity=proj[:, 7],
                rgb=proj[:, 8:11], depth32=depth32.cpu().numpy(), rect=rect, touched=touched,
                radius=radius)


def gpu_tile_lists(rast: mapping.Rasterizer):
    """(ranges[T,2], keys[I], values[I]) of the last gs_bin_sort."""
    c = rast.counters()
    I = int(c.n_instances)
    keys = rast.buffer(B.GS_BUF_TILE_KEYS, torch.int32)[:I].cpu().numpy()
    vals = rast.buffer(B.GS_BUF_TILE_VALUES, torch.int32)[:I].cpu().numpy()
    ranges = rast.buffer(B.GS_BUF_RANGES, torch.int32)[: 2 * rast.total_tiles].view(-1, 2)
    return ranges.cpu().numpy(), keys, vals, c


def guard_pixel_mask(view, proj, rout, tile=(16, 16), params=None,
                     pixel_bits=oracle.GPX_ALPHA | oracle.GPX_TRANS | oracle.GPX_POWER):
    """Pixels whose value may legitimately differ between an FP32 evaluation and
    the FP64 oracle: a per-pixel decision inside its guard band, or a pixel
    that a Gaussian with a guarded rect / depth key / cull decision reaches with
    alpha >= 1/255 (within radius + one tile of its mean, from the oracle's own
    mean and conic).  A Gaussian the oracle culls at the near plane has no
    projection to localise it with: with `params` it is projected again with
    the near plane halved, else every pixel is masked."""
    H, W = view["height"], view["width"]
    tw, th = tile
    mask = (rout["guard_px"] & pixel_bits) != 0
    flagged = np.nonzero(proj["guard"] & PIXEL_GUARDS)[0]
    for g in flagged:
        radius, (cx, cy) = proj["radius"][g], proj["mean2d"][g]
        (a, b, c), op = proj["conic"][g], proj["opacity"][g]
        if op == 0.0:
            if not proj["guard"][g] & (oracle.GUARD_NEAR | oracle.GUARD_DET):
                continue  # culled on both sides: its other guards do not matter
            if params is None:
                mask[:] = True  # culled by the near plane or determinant
                return mask
            one = {k: (v[g:g + 1] if k not in ("sh", "sh_degree") else v) for k, v in params.items()}
            one["sh"] = params["sh"][:, g:g + 1]
            pg = oracle.project(one, view, tw, th, near_z=0.5 * oracle.NEAR_Z, tight=False)
            if pg["opacity"][0] == 0.0:
                mask[:] = True  # culled for another reason: cannot localise it
                return mask
            radius, (cx, cy) = pg["radius"][0], pg["mean2d"][0]
            (a, b, c), op = pg["conic"][0], pg["opacity"][0]
        reach = int(radius) + max(tw, th)
        xa, xb = max(0, int(np.floor(cx)) - reach), min(W, int(np.ceil(cx)) + reach + 1)
        ya, yb = max(0, int(np.floor(cy)) - reach), min(H, int(np.ceil(cy)) + reach + 1)
        if xa >= xb or ya >= yb:
            continue
        yy, xx = np.mgrid[ya:yb, xa:xb]
        dx, dy = cx - xx, cy - yy
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        alpha = op * np.exp(np.minimum(power, 0.0))
        mask[ya:yb, xa:xb] |= alpha >= (1.0 / 255.0) * 0.999
    return mask


def gaussians_clear_of(mask, proj, window=5):
    """Gaussians whose every pixel with alpha >= 1/255 (bounded by the square
    of its radius around its mean) lies at least `window` pixels away from a
    masked pixel: their gradients cannot feel a guard-band decision (the
    SSIM window spreads a pixel's value over `window` pixels each way).
    Culled Gaussians count as clear."""
    H, W = mask.shape
    sat = np.zeros((H + 1, W + 1), np.int64)
    sat[1:, 1:] = np.cumsum(np.cumsum(mask.astype(np.int64), 0), 1)
    r = proj["radius"].astype(np.int64) + window + 1
    cx = np.round(proj["mean2d"][:, 0]).astype(np.int64)
    cy = np.round(proj["mean2d"][:, 1]).astype(np.int64)
    xa, xb = np.clip(cx - r, 0, W), np.clip(cx + r + 1, 0, W)
    ya, yb = np.clip(cy - r, 0, H), np.clip(cy + r + 1, 0, H)
    hits = sat[yb, xb] - sat[ya, xb] - sat[yb, xa] + sat[ya, xa]
    return (proj["tiles_touched"] == 0) | (hits == 0)


# Per-pixel decisions of a Gaussian whose FP32 outcome may differ from the
# FP64 one and whose flip changes that Gaussian's own gradient by a whole
# pixel's contribution: its alpha next to 1/255 (blended or skipped) or next
# to the 0.99 clamp (gradient passed or not).  Two guarded decisions cannot
# flip that way: the sign of the power (the conic is positive definite, so
# the exact power is <= 0 and FP32 rounding, ~1e-7 of the terms, cannot make
# it positive unless the conic's condition number reaches ~1e7 -- a mean
# that projects onto a pixel centre only gives power = 0 on both sides), and
# the transmittance cut-off (GPX_TRANS): the Gaussian that ends a pixel sits
# behind T ~ 1e-4, so the pixel's share in its gradient and its effect on
# the colour behind the others are ~1e-4 of that pixel's.
DECISION_BITS = oracle.GPX_ALPHA | oracle.GPX_KINK


def gradient_keep(params, views, renders, tile=(16, 16)):
    """The Gaussians whose parameter gradients the parity tests compare: in
    every view, clear of the pixels that a Gaussian with a guarded
    whole-Gaussian decision (rect, near plane, determinant, depth key) can
    reach, widened by the SSIM window; without a per-pixel decision of their
    own in its guard band (DECISION_BITS of the oracle's guard_g); and
    without a colour or Jacobian clamp next to its kink."""
    n = params["means"].shape[0]
    keep = np.ones(n, bool)
    for view, rout in zip(views, renders):
        proj = oracle.project(params, view, *tile)
        mask = guard_pixel_mask(view, proj, rout, tile, params=params, pixel_bits=0)
        keep &= gaussians_clear_of(mask, proj)
        keep &= (rout["guard_g"] & DECISION_BITS) == 0
        keep &= (proj["guard"] & oracle.GUARD_KINK) == 0
    return keep


def grad_errors(got, want, keep):
    """Relative L2 error per parameter group over the Gaussians in keep."""
    out = {}
    for k in want:
        a, b = ((got[k][:, keep], want[k][:, keep]) if k == "sh" else (got[k][keep], want[k][keep]))
        out[k] = rel_l2(a, b)
    return out


def grad_pixel_mask(rout):
    """Pixels whose gradient contributions cross a kink (alpha clamp)."""
    return (rout["guard_px"] & oracle.GPX_KINK) != 0


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def compare_tile_lists(keys, vals, n, o, view, tile, tile_offset=0, view_index=0):
    """End-to-end list parity of one view: the GPU's sorted instances (keys:
    global tile ids, vals: view*n + index) against the oracle's tile lists
    built from its own projection `o` (made with tight rects).  The
    Gaussians with a guarded projection decision (FWD_GUARDS) are removed
    from both sides; everything else -- which (tile, Gaussian) pairs exist
    and their order in each tile -- must be equal.  Returns (pairs compared,
    pairs removed on the oracle side)."""
    tw, th = tile
    tx, ty = oracle.tile_grid(view["width"], view["height"], tw, th)
    ostart, olst = oracle.bin_tiles(o["depth"].astype(np.float32), o["rect"], o["tiles_touched"],
                                    tx, ty, o, tile)
    otile = np.repeat(np.arange(tx * ty), np.diff(ostart))
    guarded = (o["guard"] & FWD_GUARDS) != 0
    keep_o = ~guarded[olst]
    mine = (keys >= tile_offset) & (keys < tile_offset + tx * ty)
    gk = keys[mine].astype(np.int64) - tile_offset
    gv = vals[mine].astype(np.int64)
    assert np.all(gv // n == view_index)
    gv = gv % n
    keep_g = ~guarded[gv]
    np.testing.assert_array_equal(gk[keep_g], otile[keep_o])
    np.testing.assert_array_equal(gv[keep_g], olst[keep_o])
    return int(keep_o.sum()), int((~keep_o).sum())


def tile_lists_from_gpu(ranges, vals, tile_range, n):
    """{tile: [gaussian indices]} for tiles in tile_range (view-local values)."""
    out = {}
    for t in tile_range:
        b, e = ranges[t]
        out[t] = (vals[b:e] % n).tolist() if e > b else []
    return out

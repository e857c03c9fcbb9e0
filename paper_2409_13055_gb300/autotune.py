"""Autotuner for the rasteriser's launch shape.

Picks the tile shape (8x8, 16x16, 32x8), then the number of Gaussians staged
per shared-memory batch and the pixels per thread separately for the forward
and the backward kernel, by timing the projection, binning, forward, loss and
backward of one mapping iteration on the caller's own map and views with CUDA
events (Adam is independent of these choices and is left out, so the map is
not modified).
The choice is cached in a JSON file keyed by GPU name, view sizes and a
power-of-two bucket of the map size.

The tile shape changes which pixels a Gaussian may reach (its 3-sigma rect is
counted in whole tiles), so it changes the image slightly; the batch and the
pixels per thread change only the speed.  Every tile shape is checked against
the FP64 oracle by the test-suite.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import mapping

TILES = ((8, 8), (16, 16), (32, 8))
BATCHES = (32, 64, 128, 256)
PPTS = (1, 2, 4, 8)


def cache_path():
    return os.environ.get("GS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2409_13055_gb300",
                                       "autotune.json"))


def cache_key(views, n, tight_rect=True):
    name = torch.cuda.get_device_name()
    sizes = ",".join(f"{v['width']}x{v['height']}x{v.get('channels', 3)}" for v in views)
    rects = "tight" if tight_rect else "square"
    return f"{name}|{sizes}|n2^{max(0, int(math.log2(max(1, n))))}|{rects}"


def _time_config(views, gmap, targets_packed, lam, tile, batch, ppt, iters, tight_rect=True):
    """Mean (total, forward, backward) milliseconds of project + bin + forward +
    loss + pixel adjoint + projection adjoint with one launch shape."""
    rast = mapping.fit_instance_capacity(views, gmap, tile=tile, smem_batch=batch,
                                         pixels_per_thread=ppt, smem_batch_bwd=batch,
                                         pixels_per_thread_bwd=ppt, tight_rect=tight_rect)
    m, g = gmap.gs_map(), gmap.gs_map_grad()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def once(record):
        if record:
            ev[0].record()
        rast.project(m)
        rast.bin_sort(gmap.n)
        if record:
            ev[1].record()
        rast.render_fwd()
        if record:
            ev[2].record()
        rast.loss_l1_ssim(targets_packed, lam)
        if record:
            ev[3].record()
        rast.render_bwd(m, g)
        if record:
            ev[4].record()

    for _ in range(2):
        once(False)
    tot = fwd = bwd = 0.0
    for _ in range(iters):
        once(True)
        torch.cuda.synchronize()
        tot += ev[0].elapsed_time(ev[4])
        fwd += ev[1].elapsed_time(ev[2])
        bwd += ev[3].elapsed_time(ev[4])
    return tot / iters, fwd / iters, bwd / iters


def autotune(views, gmap: mapping.GaussianMap, targets_packed, lam, iters=5, use_cache=True,
             verbose=False, tight_rect=True):
    """Returns dict(tile=(w, h), smem_batch, pixels_per_thread, smem_batch_bwd,
    pixels_per_thread_bwd, ms, timings=[...])."""
    key = cache_key(views, gmap.n, tight_rect)
    path = cache_path()
    cache = {}
    fields = ("smem_batch", "pixels_per_thread", "smem_batch_bwd", "pixels_per_thread_bwd")
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            c = cache[key]
            return dict(tile=tuple(c["tile"]), ms=c["ms"], timings=[], cached=True,
                        **{k: c[k] for k in fields})
    timings = []

    def run(tile, batch, ppt):
        t = _time_config(views, gmap, targets_packed, lam, tile, batch, ppt, iters, tight_rect)
        timings.append(dict(tile=tile, smem_batch=batch, pixels_per_thread=ppt, ms=t[0],
                            fwd_ms=t[1], bwd_ms=t[2]))
        if verbose:
            print(f"autotune {tile} batch {batch} ppt {ppt}: total {t[0]:.3f} fwd {t[1]:.3f} "
                  f"bwd {t[2]:.3f} ms")

    # stage 1: tile shape x batch at one pixel per thread, by total time
    for tile in TILES:
        for batch in BATCHES:
            run(tile, batch, 1)
    tile = min(timings, key=lambda r: r["ms"])["tile"]
    # stage 2: pixels per thread for that tile; forward and backward launch
    # shapes are chosen independently from their own stage times
    for ppt in PPTS[1:]:
        if tile[0] % ppt or (tile[0] * tile[1] // ppt) % 32:
            continue
        for batch in BATCHES:
            run(tile, batch, ppt)
    mine = [r for r in timings if r["tile"] == tile]
    f = min(mine, key=lambda r: r["fwd_ms"])
    b = min(mine, key=lambda r: r["bwd_ms"])
    base = min(mine, key=lambda r: r["ms"])
    est = base["ms"] - base["fwd_ms"] - base["bwd_ms"] + f["fwd_ms"] + b["bwd_ms"]
    out = dict(tile=tile, smem_batch=f["smem_batch"], pixels_per_thread=f["pixels_per_thread"],
               smem_batch_bwd=b["smem_batch"], pixels_per_thread_bwd=b["pixels_per_thread"],
               ms=est, timings=timings, cached=False)
    if use_cache:
        cache[key] = dict(tile=list(tile), ms=est, **{k: out[k] for k in fields})
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(cache, fh, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return out

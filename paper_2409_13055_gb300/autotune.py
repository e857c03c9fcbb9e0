"""Autotuner for the rasteriser's launch shape.

Picks the tile shape (8x8, 16x16, 32x8), the number of Gaussians staged per
shared-memory batch and the pixels per thread by timing the forward, loss and
backward of one mapping iteration on the caller's own map and views (Adam is
independent of these choices and is left out, so the map is not modified).
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
BATCHES = (32, 64, 128)
PPTS = (1, 2)


def cache_path():
    return os.environ.get("GS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2409_13055_gb300",
                                       "autotune.json"))


def cache_key(views, n):
    name = torch.cuda.get_device_name()
    sizes = ",".join(f"{v['width']}x{v['height']}x{v.get('channels', 3)}" for v in views)
    return f"{name}|{sizes}|n2^{max(0, int(math.log2(max(1, n))))}"


def _time_config(views, gmap, targets_packed, lam, tile, batch, ppt, iters):
    rast = mapping.fit_instance_capacity(views, gmap, tile=tile, smem_batch=batch,
                                         pixels_per_thread=ppt)
    m, g = gmap.gs_map(), gmap.gs_map_grad()

    def once():
        rast.project(m)
        rast.bin_sort(gmap.n)
        rast.render_fwd()
        rast.loss_l1_ssim(targets_packed, lam)
        rast.render_bwd(m, g)

    for _ in range(2):
        once()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(iters):
        once()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / iters


def autotune(views, gmap: mapping.GaussianMap, targets_packed, lam, iters=5, use_cache=True,
             verbose=False):
    """Returns dict(tile=(w, h), smem_batch=b, pixels_per_thread=p, ms=t, timings=[...])."""
    key = cache_key(views, gmap.n)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            c = cache[key]
            return dict(tile=tuple(c["tile"]), smem_batch=c["smem_batch"],
                        pixels_per_thread=c["pixels_per_thread"], ms=c["ms"], timings=[],
                        cached=True)
    timings = []
    # stage 1: tile shape x batch at one pixel per thread
    for tile in TILES:
        for batch in BATCHES:
            t = _time_config(views, gmap, targets_packed, lam, tile, batch, 1, iters)
            timings.append((t, tile, batch, 1))
            if verbose:
                print(f"autotune {tile} batch {batch} ppt 1: {t:.3f} ms")
    best = min(timings)
    # stage 2: more pixels per thread at the best tile and batch
    for ppt in PPTS[1:]:
        tile, batch = best[1], best[2]
        if tile[0] % ppt or (tile[0] * tile[1] // ppt) % 32:
            continue
        t = _time_config(views, gmap, targets_packed, lam, tile, batch, ppt, iters)
        timings.append((t, tile, batch, ppt))
        if verbose:
            print(f"autotune {tile} batch {batch} ppt {ppt}: {t:.3f} ms")
    best = min(timings)
    out = dict(tile=best[1], smem_batch=best[2], pixels_per_thread=best[3], ms=best[0],
               timings=[dict(ms=t, tile=tl, smem_batch=b, pixels_per_thread=p)
                        for (t, tl, b, p) in timings], cached=False)
    if use_cache:
        cache[key] = dict(tile=list(out["tile"]), smem_batch=out["smem_batch"],
                          pixels_per_thread=out["pixels_per_thread"], ms=out["ms"])
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return out

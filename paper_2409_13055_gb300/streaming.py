"""Streaming mapping: keyframes arrive one at a time, each inserting new
Gaussians, and the map is optimised over a sliding window of the latest
keyframes (paper Sec. III-B: the mapping thread receives keyframes and the
photometric-SLAM point cloud, initialises Gaussians from it and optimises them
over a window of keyframes).

Per keyframe:
  1. its new Gaussians are appended to the map (``GaussianMap.append``: Adam
     moments zero, step counter kept);
  2. the window's views, targets and rasteriser are set up (one rasteriser,
     planned for the window size and the map's capacity and re-planned with
     headroom when either changes or the instance count outgrows it);
  3. ``iters`` batched mapping iterations run over the whole window, each one
     ``MappingStep`` (project, bin, render, loss, backward, Adam), by default
     on a recompute rasteriser (checkpointing: the window's views go through a
     workspace of four views a pass at a time, and the backward repeats each
     pass's projection and binning), captured as one CUDA graph and replayed;
     with Gaussian-pyramid targets (Sec. III-B) the iterations go from the
     coarsest level to the full resolution.

Every arithmetic step runs in libgs_gb300.so; this module only moves memory
and decides when to re-plan.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mapping, pyramid


class StreamingMapper:
    """Sliding-window mapper over a growing map, optionally with
    Gaussian-pyramid targets (``pyramid_levels`` > 1: each keyframe's
    iterations run coarse to fine, see ``pyramid.level_for``)."""

    def __init__(self, degree=3, window=8, iters=30, lam=0.2, lr=None, extent=1.0,
                 recompute=4, capacity=1 << 20, instance_headroom=1.25, graphs=True,
                 pyramid_levels=1, device="cuda", **rast_kw):
        # recompute: views per pass of the checkpointing rasteriser (True:
        # 1, False/0: none, every view's projection kept)
        self.degree, self.window, self.iters, self.lam = int(degree), int(window), int(iters), lam
        self.lr, self.extent, self.recompute = lr, extent, int(recompute)
        self.capacity, self.headroom, self.graphs = int(capacity), float(instance_headroom), graphs
        self.levels = max(1, int(pyramid_levels))
        self.device = torch.device(device)
        self.rast_kw = rast_kw
        self.gmap = None
        self.frames = []        # (view, target) of the window, oldest first
        self._rasts = {}        # (window size, level) -> Rasterizer (current size only)
        self.steps = []         # MappingStep per pyramid level
        self.keyframes = 0
        self.iterations = 0
        self.replans = 0

    # -- set-up ---------------------------------------------------------------
    def _rasterizer(self, views, level):
        V = len(views)
        key = (V, level)
        r = self._rasts.get(key)
        n = self.gmap.n
        if r is None or r.n_capacity < n:
            while self.capacity < n:
                self.capacity *= 2
            r = mapping.Rasterizer(views, self.capacity, instance_capacity=None,
                                   recompute=self.recompute, **self.rast_kw)
            # a smaller window does not come back once the window is full, and
            # each plan's workspace grows with views x capacity
            self._rasts = {k: v for k, v in self._rasts.items() if k[0] == V}
            self._rasts[key] = r
            self.replans += 1
        r.set_poses(views)
        # instance capacity (of a view, in a recompute plan): one synchronising
        # probe per keyframe, level and pass
        raw = r.max_instances(self.gmap.gs_map())
        if raw > r.instance_capacity:
            r = mapping.Rasterizer(views, self.capacity,
                                   instance_capacity=int(raw * self.headroom) + 4096,
                                   recompute=self.recompute, **self.rast_kw)
            r.set_poses(views)
            self._rasts[key] = r
            self.replans += 1
        return r

    def insert_keyframe(self, view, target, new_gaussians):
        """Append the keyframe's Gaussians, slide the window and prepare the
        window's mapping iteration at every pyramid level (not yet run)."""
        if self.gmap is None:
            self.gmap = mapping.GaussianMap(new_gaussians, self.device)
        else:
            self.gmap.append(new_gaussians)
        tgt = torch.as_tensor(np.asarray(target, np.float32)).to(self.device)
        self.frames.append((view, pyramid.pyramid(tgt, self.levels)))
        if len(self.frames) > self.window:
            self.frames.pop(0)
        self.steps = []
        for level in range(self.levels):
            views = [pyramid.level_view(f[0], level) for f in self.frames]
            rast = self._rasterizer(views, level)
            targets = torch.cat([f[1][level].reshape(-1) for f in self.frames])
            self.steps.append(mapping.MappingStep(self.gmap, rast, targets, self.lam, self.lr,
                                                  self.extent))
        self._eager_done = [False] * self.levels
        self._kf_iter = 0
        self.keyframes += 1

    @property
    def step(self):
        """The MappingStep of the level the next iteration uses."""
        return self.steps[pyramid.level_for(self._kf_iter, self.iters, self.levels)]

    def iterate(self, k=1):
        """k mapping iterations over the current window, each at the level of
        the coarse-to-fine schedule: a level's first iteration runs eagerly,
        the rest replay a graph captured after it."""
        for _ in range(k):
            level = pyramid.level_for(self._kf_iter, self.iters, self.levels)
            step = self.steps[level]
            if self.graphs and step.graph is None and self._eager_done[level]:
                step.capture(warmup=0)
            step()
            self.last_step = step
            self._eager_done[level] = True
            self._kf_iter += 1
            self.iterations += 1

    def add_keyframe(self, view, target, new_gaussians):
        """One keyframe of the mapping thread: insert it (window, new
        Gaussians, replan if needed), then run this mapper's iterations."""
        self.insert_keyframe(view, target, new_gaussians)
        self.iterate(self.iters)

    def status(self):
        """Device status of the finest level's rasteriser (synchronises)."""
        return self.steps[0].rast.counters()

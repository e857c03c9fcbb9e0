"""Point-cloud densification for new keyframes (paper Sec. III-A): DSO-style
pixel selection, then points in flat regions at the mean depth of the
vertices of their triangle in the Delaunay triangulation of the tracked
pixels, then new Gaussians from the points (the map's insertion of Sec.
III-B).

* ``select_pixels`` -- GPU (``gs_select_pixels``): squared gradient and the
  pass of each selected pixel;
* ``triangulate`` -- host (``gs_delaunay``), exact integer predicates;
* ``interpolate`` -- GPU (``gs_interp_depth``): depths of the flat grid
  pixels;
* ``keyframe_points`` -- the three steps for one keyframe, given the depth
  the tracker assigns to each selected pixel;
* ``gaussians_from_points`` -- the new Gaussians: back-projected means,
  isotropic scale of ``footprint_px`` pixels at their depth, identity
  rotation, opacity 0.1, SH DC from the pixel's gray value.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B

DEFAULT_THRESHOLDS_SQ = (4.0e-4, 2.25e-4, 1.0e-4)  # (0.02, 0.015, 0.01)^2 per pass


def select_pixels(gray: torch.Tensor, block=4, thresholds_sq=DEFAULT_THRESHOLDS_SQ, stream=None):
    gray = gray.contiguous()
    H, W = gray.shape
    g2 = torch.empty((H, W), dtype=torch.float32, device=gray.device)
    sel = torch.empty((H, W), dtype=torch.int32, device=gray.device)
    B.gs_select_pixels(gray, block, thresholds_sq, g2, sel, stream)
    return g2, sel


def triangulate(xy: np.ndarray) -> np.ndarray:
    return B.gs_delaunay(xy)


def interpolate(tri: torch.Tensor, xy: torch.Tensor, depth: torch.Tensor, g2: torch.Tensor,
                sel: torch.Tensor, grid=4, flat_sq=1.0e-4, stream=None) -> torch.Tensor:
    H, W = g2.shape
    gh, gw = (H + grid - 1) // grid, (W + grid - 1) // grid
    owner = torch.empty((gh, gw), dtype=torch.int32, device=g2.device)
    out = torch.empty((gh, gw), dtype=torch.float32, device=g2.device)
    B.gs_interp_depth(tri, xy, depth, g2, sel, grid, flat_sq, owner, out, stream)
    return out


def keyframe_points(gray: torch.Tensor, depth_of, block=4, thresholds_sq=DEFAULT_THRESHOLDS_SQ,
                    grid=4, flat_sq=1.0e-4):
    """(px, py, z) of the tracked and the interpolated points of a keyframe.
    depth_of(px, py) -> depths of the selected pixels (the tracker's
    estimates).  One host round trip for the selected pixels."""
    g2, sel = select_pixels(gray, block, thresholds_sq)
    ys, xs = torch.nonzero(sel, as_tuple=True)  # raster order
    z = depth_of(xs, ys).to(torch.float32)
    xy = torch.stack([xs, ys], 1).to(torch.int32)
    tri = torch.as_tensor(triangulate(xy.cpu().numpy()), device=gray.device)
    if tri.numel() == 0:
        return xs, ys, z
    fz = interpolate(tri.contiguous(), xy.contiguous(), z.contiguous(), g2, sel, grid, flat_sq)
    gy, gx = torch.nonzero(fz, as_tuple=True)
    return (torch.cat([xs, gx * grid]), torch.cat([ys, gy * grid]), torch.cat([z, fz[gy, gx]]))


def gaussians_from_points(view, px, py, z, gray: torch.Tensor, sh_degree=3, footprint_px=2.0,
                          opacity=0.1):
    """New Gaussians (host numpy dict in the map layout) at the back-projected
    points: isotropic log-scale log(z footprint / fx), identity rotation, the
    given opacity, SH DC (gray - 0.5) / Y00 on all three channels."""
    dev = gray.device
    R = torch.as_tensor(np.asarray(view["R"], np.float32), device=dev)
    t = torch.as_tensor(np.asarray(view["t"], np.float32), device=dev)
    x = (px.to(torch.float32) - view["cx"]) / view["fx"] * z
    y = (py.to(torch.float32) - view["cy"]) / view["fy"] * z
    xc = torch.stack([x, y, z], 1)
    means = (xc - t) @ R  # R^T (x_c - t)
    n = means.shape[0]
    K = (sh_degree + 1) ** 2
    sh = torch.zeros((K, n, 3), device=dev)
    sh[0] = ((gray[py, px] - 0.5) * (2.0 * math.sqrt(math.pi))).unsqueeze(1)
    q = torch.zeros((n, 4), device=dev)
    q[:, 0] = 1.0
    ls = torch.log(z * (footprint_px / view["fx"])).unsqueeze(1).expand(n, 3)
    return dict(means=means.cpu().numpy(), log_scales=ls.contiguous().cpu().numpy(),
                quats=q.cpu().numpy(),
                opacity_logits=np.full(n, math.log(opacity / (1 - opacity)), np.float32),
                sh=sh.cpu().numpy(), sh_degree=sh_degree)

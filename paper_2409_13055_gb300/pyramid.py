"""Gaussian-pyramid targets for progressive training (paper Sec. III-B: the
keyframe image is smoothed and down-sampled repeatedly; the loss starts on
the coarsest level and moves to finer ones as training advances).

* ``pyr_down`` -- one level on the GPU (``gs_pyr_down``: binomial 5x5,
  mirrored borders, every second pixel);
* ``level_view`` -- the camera of level L (half the focal lengths and
  principal point per level, ceil-halved sizes), under which pixel i of
  level L+1 is pixel 2i of level L;
* ``level_for`` -- the coarse-to-fine schedule: the iterations of a keyframe
  are split into ``levels`` equal runs, coarsest first.
"""
from __future__ import annotations

import torch

from . import binding as B


def level_view(view, level):
    v = dict(view)
    for _ in range(int(level)):
        v = dict(v, width=(v["width"] + 1) // 2, height=(v["height"] + 1) // 2,
                 fx=v["fx"] / 2, fy=v["fy"] / 2, cx=v["cx"] / 2, cy=v["cy"] / 2)
    return v


def pyr_down(img: torch.Tensor, stream=None) -> torch.Tensor:
    """[C][H][W] float32 CUDA tensor -> [C][ceil(H/2)][ceil(W/2)]."""
    C, H, W = img.shape
    out = torch.empty((C, (H + 1) // 2, (W + 1) // 2), dtype=torch.float32, device=img.device)
    B.gs_pyr_down(img.contiguous(), C, H, W, out, stream)
    return out


def pyramid(img: torch.Tensor, levels: int, stream=None):
    """[level 0 = img, level 1, ..., level levels-1]."""
    out = [img]
    for _ in range(int(levels) - 1):
        out.append(pyr_down(out[-1], stream))
    return out


def level_for(iteration: int, iters: int, levels: int) -> int:
    """Pyramid level of iteration `iteration` (0-based) of `iters`."""
    if levels <= 1 or iters <= 0:
        return 0
    return max(0, levels - 1 - (iteration * levels) // iters)

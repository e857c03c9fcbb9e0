"""Writes tests/golden/oracle_small.json from the FP64 oracle alone.

The paper prints no worked example for the rasteriser, so this fixture is an
oracle regression record, not a pin: it freezes the oracle's outputs on one
small seeded scene (40 Gaussians, SH degree 3, 32x24, a rotated camera, L1+SSIM
with lambda = 0.2) so that any later change to the oracle's arithmetic shows
up as a failing test and has to be justified.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2409_13055_gb300 import scenes  # noqa: E402


def golden_case():
    p, view = scenes.tiny_scene(40, 32, 24, seed=77, sh_degree=3)
    R, t = scenes.random_pose(np.random.default_rng(78), 0.2, 15.0)
    view = dict(view, R=R, t=t * 0.1)
    target = scenes.random_target(view, 79)
    return p, view, target


def compute(tight=False):
    """The record is of the plain 3-sigma square tile rects (tight=False)."""
    p, view, target = golden_case()
    L, g, renders = oracle.iteration(p, [view], [target], 0.2, bg=(0.1, 0.2, 0.3), tight=tight)
    img = renders[0]["image"]
    rng = np.random.default_rng(80)
    pix = [(int(c), int(y), int(x)) for c, y, x in
           zip(rng.integers(0, 3, 48), rng.integers(0, 24, 48), rng.integers(0, 32, 48))]
    return {
        "loss": L,
        "image_sum": float(img.sum()),
        "final_T_sum": float(renders[0]["final_T"].sum()),
        "last_idx_sum": int(renders[0]["last_idx"].sum()),
        "pixels": [[c, y, x, float(img[c, y, x])] for c, y, x in pix],
        "grad_norms": {k: float(np.linalg.norm(v)) for k, v in g.items()},
        "grad_means_first": [float(v) for v in g["means"][:4].ravel()],
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", out)

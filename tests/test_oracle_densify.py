"""Pins of the oracle's adaptive density control (paper Sec. III-B: densify
Gaussians with a high homodirectional view-space position gradient -- the
AbsGS criterion -- by cloning small ones and splitting large ones with the
original 3DGS parameters, and prune low-opacity ones).

References used: the statistic rebuilt pixel by pixel from the (separately
pinned) compositing adjoint with the loss gradient restricted to one pixel;
the triangle inequality and its equality case; the NDC change of variables;
hand-built categories; an explicit rotation matrix for the split offsets.
"""
import math

import numpy as np

import oracle
from paper_2409_13055_gb300 import scenes


def _scene():
    p, view = scenes.tiny_scene(12, 24, 16, seed=7, sh_degree=1)
    return p, view


def test_homodirectional_gradient_is_the_sum_of_per_pixel_magnitudes():
    """dmean2d_abs equals the sum over pixels of |d L_p / d mean2d|, where L_p
    keeps only pixel p's part of the loss gradient, each such adjoint being the
    compositing adjoint already pinned by finite differences."""
    p, view = _scene()
    W, H = view["width"], view["height"]
    proj, st, lst, out = oracle.forward_view(p, view, 8, 8)
    rng = np.random.default_rng(3)
    dimg = rng.normal(size=(3, H, W))
    full = oracle.render_bwd(proj, st, lst, view, dimg, 8, 8)
    acc = np.zeros_like(full["dmean2d"])
    for y in range(H):
        for x in range(W):
            d = np.zeros_like(dimg)
            d[:, y, x] = dimg[:, y, x]
            acc += np.abs(oracle.render_bwd(proj, st, lst, view, d, 8, 8)["dmean2d"])
    np.testing.assert_allclose(full["dmean2d_abs"], acc, rtol=1e-12, atol=1e-15)
    assert np.all(full["dmean2d_abs"] + 1e-15 >= np.abs(full["dmean2d"]))
    assert np.any(full["dmean2d_abs"] > 1.01 * np.abs(full["dmean2d"]))


def test_homodirectional_equals_plain_when_contributions_share_a_sign():
    """One isotropic Gaussian left of the image, positive colour, dL/dC = 1,
    black background: every pixel sees dx < 0, b = 0 and the same sign of
    dL/dalpha, so every x-contribution has one sign and |sum| = sum |.|."""
    W, H, f = 20, 12, 30.0
    view = scenes.camera(W, H, f, f, 10.0, 6.0)
    y00 = 0.5 / math.sqrt(math.pi)
    z = 2.0
    mx = (-3.0 - 10.0) / f * z  # projected mean at x = -3 px, y = 6 px
    p = dict(means=np.array([[mx, 0.0, z]]), log_scales=np.full((1, 3), math.log(0.2)),
             quats=np.array([[1.0, 0, 0, 0]]), opacity_logits=np.array([1.0]),
             sh=((np.array([0.8, 0.6, 0.7]) - 0.5) / y00).reshape(1, 1, 3), sh_degree=0)
    proj, st, lst, out = oracle.forward_view(p, view, 4, 4)
    assert abs(proj["conic"][0, 1]) < 1e-12
    g = oracle.render_bwd(proj, st, lst, view, np.ones((3, H, W)), 4, 4)
    assert g["dmean2d_abs"][0, 0] > 0
    assert math.isclose(g["dmean2d_abs"][0, 0], abs(g["dmean2d"][0, 0]), rel_tol=1e-12)


def test_stats_use_ndc_units_and_count_visible_views():
    view = dict(width=200, height=100)
    accum, denom = np.zeros(3), np.zeros(3)
    abs2 = np.array([[1e-6, 2e-6], [3e-6, 0.0], [5.0, 5.0]])
    oracle.densify_stats(accum, denom, view, np.array([1, 4, 0]), abs2)
    oracle.densify_stats(accum, denom, view, np.array([2, 0, 0]), abs2)
    np.testing.assert_allclose(accum[:2], [2 * math.hypot(100e-6, 100e-6), 300e-6], rtol=1e-14)
    np.testing.assert_array_equal(denom, [2, 1, 0])
    assert accum[2] == 0


def _five():
    # opacity logit, log-scales, accum, denom -> expected category
    rows = [(-6.0, -5.0, 1.0, 1.0, oracle.PRUNE),      # opacity 0.0025 < 0.005
            (0.0, -5.0, 1e-4, 1.0, oracle.KEEP),       # statistic below 4e-4
            (0.0, -5.0, 9e-4, 2.0, oracle.CLONE),      # 4.5e-4, scale 6.7e-3 <= 0.01
            (0.0, -4.0, 9e-4, 2.0, oracle.SPLIT),      # 4.5e-4, scale 1.8e-2 > 0.01
            (0.0, -4.0, 1.0, 0.0, oracle.KEEP)]        # never visible
    n = len(rows)
    p = dict(means=np.arange(3 * n, dtype=float).reshape(n, 3),
             log_scales=np.array([[r[1], r[1] - 1.0, r[1] - 2.0] for r in rows]),
             quats=np.tile([1.0, 0, 0, 0], (n, 1)),
             opacity_logits=np.array([r[0] for r in rows]),
             sh=np.arange(4 * n * 3, dtype=float).reshape(4, n, 3), sh_degree=1)
    return p, np.array([r[2] for r in rows]), np.array([r[3] for r in rows]), \
        np.array([r[4] for r in rows])


def test_categories_follow_opacity_statistic_and_size():
    p, accum, denom, want = _five()
    np.testing.assert_array_equal(oracle.densify_categories(p, accum, denom, extent=1.0), want)
    # pruning takes precedence over a high statistic
    p["opacity_logits"][2] = -7.0
    assert oracle.densify_categories(p, accum, denom, 1.0)[2] == oracle.PRUNE


def test_apply_order_clones_children_and_moments():
    p, accum, denom, _ = _five()
    p["quats"][3] = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]  # 90 deg about z
    cat = oracle.densify_categories(p, accum, denom, 1.0)
    samples = np.zeros((5, 2, 3))
    samples[3] = [[1.0, 0.0, 0.0], [0.0, 2.0, -1.0]]
    mom = {k: (np.full_like(np.asarray(p[k], float), 1.5), np.full_like(np.asarray(p[k], float), 2.5))
           for k in oracle.PARAM_GROUPS}
    out, nm = oracle.densify_apply(p, mom, cat, samples)
    # kept: 1, 2, 4; clone of 2; children of 3
    order = [1, 2, 4, 2, 3, 3]
    assert out["means"].shape == (6, 3)
    np.testing.assert_array_equal(out["opacity_logits"], p["opacity_logits"][order])
    np.testing.assert_array_equal(out["quats"], p["quats"][order])
    np.testing.assert_array_equal(out["sh"], p["sh"][:, order])
    np.testing.assert_array_equal(out["means"][:4], p["means"][[1, 2, 4, 2]])
    np.testing.assert_array_equal(out["log_scales"][:4], p["log_scales"][[1, 2, 4, 2]])
    # children: mean + R (s * xi) with R = rotation by 90 degrees about z
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    s = np.exp(p["log_scales"][3])
    for c in range(2):
        np.testing.assert_allclose(out["means"][4 + c], p["means"][3] + Rz @ (s * samples[3, c]),
                                   atol=1e-12)
        np.testing.assert_allclose(out["log_scales"][4 + c], p["log_scales"][3] - math.log(1.6),
                                   atol=1e-15)
    for k, (m, v) in nm.items():
        ax = 1 if k == "sh" else 0
        kept = np.take(m, [0, 1, 2], axis=ax)
        new = np.take(m, [3, 4, 5], axis=ax)
        assert np.all(kept == 1.5) and np.all(new == 0) and np.all(np.take(v, [3, 4, 5], axis=ax) == 0)

"""Pins of the oracle's photometric loss (Eq. 2, read as
L = (1-lambda) mean|I - I_gt| + lambda (1 - mean SSIM)), its Adam step
(Sec. IV-A: the default 3DGS optimiser) and the whole mapping iteration.

References: the SSIM of Wang et al. rebuilt from scipy.ndimage correlations
and scipy's Gaussian window; closed forms for identical and constant images;
torch.optim.Adam in float64; central differences of the loss and of the full
render-loss pipeline.
"""
import math

import numpy as np
import pytest
import torch
from scipy import ndimage
from scipy.signal import windows

import oracle
from paper_2409_13055_gb300 import scenes


def test_window_is_normalised_gaussian():
    g = windows.gaussian(11, 1.5)
    g = g / g.sum()
    np.testing.assert_allclose(oracle.ssim_window(), np.outer(g, g), rtol=1e-14)


def ssim_map_scipy(x, y):
    g = windows.gaussian(11, 1.5)
    g = np.outer(g, g) / g.sum() ** 2
    f = lambda a: ndimage.correlate(a, g, mode="constant", cval=0.0)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    mx, my = f(x), f(y)
    vx, vy, cxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))


@pytest.mark.parametrize("shape", [(3, 20, 27), (1, 13, 9)])
def test_ssim_matches_scipy_construction(shape):
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 1, shape), rng.uniform(0, 1, shape)
    lam = 0.2
    L, _, smap = oracle.loss_l1_ssim(x, y, lam, want_map=True)
    want_map = np.stack([ssim_map_scipy(x[c], y[c]) for c in range(shape[0])])
    np.testing.assert_allclose(smap, want_map, rtol=1e-12, atol=1e-14)
    want = (1 - lam) * np.abs(x - y).mean() + lam * (1 - want_map.mean())
    assert abs(L - want) < 1e-13


def test_identical_images_zero_loss_and_gradient():
    x = np.random.default_rng(1).uniform(0, 1, (3, 16, 16))
    L, d = oracle.loss_l1_ssim(x, x, 0.2)
    assert abs(L) < 1e-14
    assert np.abs(d).max() < 1e-14


def test_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    x, y = np.full((1, 30, 30), a), np.full((1, 30, 30), b)
    _, _, smap = oracle.loss_l1_ssim(x, y, 1.0, want_map=True)
    C1 = 0.01 ** 2
    np.testing.assert_allclose(smap[0, 5:-5, 5:-5], (2 * a * b + C1) / (a * a + b * b + C1),
                               rtol=1e-12)
    L, _ = oracle.loss_l1_ssim(x, y, 0.0)
    assert abs(L - 0.4) < 1e-13


@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_loss_gradient_central_differences(lam):
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, (3, 9, 11)), rng.uniform(0, 1, (3, 9, 11))
    L, d = oracle.loss_l1_ssim(x, y, lam)
    h = 1e-6
    flat = x.reshape(-1)
    for j in range(flat.size):
        old = flat[j]
        flat[j] = old + h
        Lp, _ = oracle.loss_l1_ssim(x, y, lam, want_grad=False)
        flat[j] = old - h
        Lm, _ = oracle.loss_l1_ssim(x, y, lam, want_grad=False)
        flat[j] = old
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - d.reshape(-1)[j]) < 1e-8, (j, fd, d.reshape(-1)[j])


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=100)
    g = rng.normal(size=100)
    g[:5] = 0.0
    p, m, v = p0.copy(), np.zeros(100), np.zeros(100)
    oracle.adam(p, g, m, v, lr=0.01, step=1)
    np.testing.assert_allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-15), rtol=1e-14, atol=1e-16)
    assert np.array_equal(p[:5], p0[:5])


def test_adam_matches_torch_float64():
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=200)
    tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(200), np.zeros(200)
    for step in range(1, 6):
        g = rng.normal(size=200) * (0.1 ** step)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        oracle.adam(p, g, m, v, lr=3e-3, step=step)
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------------------
# The whole mapping iteration: central differences through project, bin,
# render and loss (h = 1e-6), skipping perturbations that flip a decision.
# ----------------------------------------------------------------------------
def _decisions(renders):
    return [np.concatenate([r["last_idx"].ravel(), r["n_eval"].ravel(), r["n_included"].ravel()])
            for r in renders]


@pytest.mark.parametrize("degree,lam,channels", [(0, 0.0, 3), (3, 0.2, 3), (1, 0.2, 1)])
def test_iteration_gradient_central_differences(degree, lam, channels):
    n = 10
    p, view = scenes.tiny_scene(n, 24, 20, seed=30 + degree, sh_degree=degree)
    p = {k: (v.astype(float) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    rng = np.random.default_rng(5)
    R, t = scenes.random_pose(rng, 0.2, 10.0)
    view = dict(view, R=R.astype(float), t=t.astype(float) * 0.1, channels=channels)
    view2 = dict(view, t=np.asarray(view["t"]) + np.array([0.05, 0.0, 0.02]))
    views = [view, view2]
    targets = [rng.uniform(0, 1, (channels, 20, 24)) for _ in views]
    L, g, renders = oracle.iteration(p, views, targets, lam, bg=(0.1, 0.2, 0.3))
    base_dec = _decisions(renders)
    h = 1e-6
    checked = total = 0
    for key in oracle.PARAM_GROUPS:
        flat = p[key].reshape(-1)
        gflat = g[key].reshape(-1)
        for j in range(flat.size):
            total += 1
            old = flat[j]
            flat[j] = old + h
            Lp, _, rp = oracle.iteration(p, views, targets, lam, bg=(0.1, 0.2, 0.3))
            flat[j] = old - h
            Lm, _, rm = oracle.iteration(p, views, targets, lam, bg=(0.1, 0.2, 0.3))
            flat[j] = old
            if not all(np.array_equal(a, b) and np.array_equal(a, c)
                       for a, b, c in zip(base_dec, _decisions(rp), _decisions(rm))):
                continue
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - gflat[j]) <= 1e-6 + 1e-5 * abs(fd), (key, j, fd, gflat[j])
            checked += 1
    assert checked > 0.9 * total


def test_masked_adam_equals_dense_on_its_elements_and_leaves_the_rest():
    """All-true mask = the dense step bit for bit; false entries unchanged."""
    rng = np.random.default_rng(12)
    n = 50
    p0, g, m0, v0 = rng.normal(size=n), rng.normal(size=n), rng.normal(size=n), rng.uniform(size=n)
    a = [x.copy() for x in (p0, m0, v0)]
    b = [x.copy() for x in (p0, m0, v0)]
    oracle.adam(a[0], g, a[1], a[2], 1e-3, 3)
    oracle.adam_masked(b[0], g, b[1], b[2], 1e-3, 3, np.ones(n, bool))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    mask = rng.uniform(size=n) < 0.4
    c = [x.copy() for x in (p0, m0, v0)]
    oracle.adam_masked(c[0], g, c[1], c[2], 1e-3, 3, mask)
    for x, y, z in zip(c, a, (p0, m0, v0)):
        np.testing.assert_array_equal(x[mask], y[mask])
        np.testing.assert_array_equal(x[~mask], z[~mask])


def test_room200k_subset_gradient_central_differences():
    """The 200k-Gaussian room at 640x480 (f = 525; anisotropic, SH degree 3,
    L1 + 0.2 (1 - SSIM)): on a subset of 64 of its Gaussians, those whose
    means project nearest the image centre, rendered through a 48x40 crop of
    the same camera, the oracle's analytic gradient against central
    differences (h = 1e-6) of its whole iteration: along a random direction
    of every parameter group of every Gaussian, and coordinate by coordinate
    for 8 of them; perturbations that flip a decision are skipped."""
    p_all, views, targets, lam = scenes.workload("room200k_640x480")
    full = views[0]
    pr = oracle.project(p_all, full, 16, 16, tight=False)
    vis = np.flatnonzero(pr["tiles_touched"] > 0)
    d = np.hypot(pr["mean2d"][vis, 0] - 320.0, pr["mean2d"][vis, 1] - 240.0)
    idx = np.sort(vis[np.argsort(d)[:64]])
    p = scenes.subset(p_all, idx)
    p = {k: (v.astype(float) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    W, H = 48, 40
    view = scenes.camera(W, H, 525.0, 525.0, cx=320.0 - 296.0, cy=240.0 - 220.0)
    target = np.asarray(targets[0], float)[:, 220:220 + H, 296:296 + W]
    L, g, renders = oracle.iteration(p, [view], [target], lam)
    assert (renders[0]["n_included"] > 0).mean() > 0.5  # the subset covers the crop
    base = _decisions(renders)
    h = 1e-6
    rng = np.random.default_rng(64)

    def loss_at(key, j, delta):
        flat = p[key].reshape(-1)
        old = flat[j].copy()
        flat[j] = old + delta
        Lx, _, r = oracle.iteration(p, [view], [target], lam)
        flat[j] = old
        return Lx, _decisions(r)

    checked = total = 0
    for i in range(64):
        for key in oracle.PARAM_GROUPS:
            # the coordinates of Gaussian i in this group
            j = (np.arange(p["sh"].shape[0])[:, None] * 64 * 3 + i * 3 + np.arange(3)).ravel() \
                if key == "sh" else np.arange(p[key][i].size) + i * p[key][i].size
            coords = [(j, rng.normal(size=j.size))] + ([(np.array([k]), np.ones(1)) for k in j]
                                                       if i < 8 else [])
            for jj, u in coords:
                u = u / np.linalg.norm(u)
                total += 1
                Lp, dp = loss_at(key, jj, h * u)
                Lm, dm = loss_at(key, jj, -h * u)
                if not all(np.array_equal(a, b) and np.array_equal(a, c)
                           for a, b, c in zip(base, dp, dm)):
                    continue
                fd = (Lp - Lm) / (2 * h)
                an = float(np.dot(g[key].reshape(-1)[jj], u))
                assert abs(fd - an) <= 1e-7 + 1e-5 * abs(fd), (i, key, jj, fd, an)
                checked += 1
    assert checked > 0.9 * total, (checked, total)

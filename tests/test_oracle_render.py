"""Pins of the oracle's binning, compositing and compositing adjoint
(Sec. II: depth sorting and front-to-back blending; Sec. III-B: the original
3DGS tile-based rasteriser).

References used: closed forms for one isotropic Gaussian, the telescoping
transmittance identity, brute force without tile lists, numpy's lexsort,
permutation invariance, linearity of grayscale, and central differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_13055_gb300 import scenes


def one_gaussian(mean, log_s, logit, rgb):
    y00 = 0.5 / math.sqrt(math.pi)
    sh = ((np.asarray(rgb, float) - 0.5) / y00).reshape(1, 1, 3)
    return dict(means=np.array([mean], float), log_scales=np.full((1, 3), log_s),
                quats=np.array([[1.0, 0, 0, 0]]), opacity_logits=np.array([logit]), sh=sh,
                sh_degree=0)


def test_single_isotropic_gaussian_closed_form():
    W, H, f = 64, 48, 80.0
    view = scenes.camera(W, H, f, f, 31.3, 22.6)
    z, s, logit = 1.5, 0.03, 1.2
    rgb = [0.9, 0.2, 0.4]
    bg = (0.1, 0.3, 0.5)
    p = one_gaussian([0.02, -0.01, z], math.log(s), logit, rgb)
    proj, st, lst, out = oracle.forward_view(p, view, bg=bg)
    o = 1 / (1 + math.exp(-logit))
    # isotropic Sigma = s^2 I seen off-axis: Sigma' = s^2 J J^T + 0.3 I (pinhole J)
    x, y = 0.02, -0.01
    J = np.array([[f / z, 0, -f * x / z ** 2], [0, f / z, -f * y / z ** 2]])
    cov = s * s * J @ J.T + 0.3 * np.eye(2)
    Q = np.linalg.inv(cov)
    mu = np.array([f * x / z + 31.3, f * y / z + 22.6])
    r = math.ceil(3 * math.sqrt(np.linalg.eigvalsh(cov).max()))
    tx0, ty0 = max(0, math.floor((mu[0] - r) / 16)), max(0, math.floor((mu[1] - r) / 16))
    tx1, ty1 = min(4, math.floor((mu[0] + r + 15) / 16)), min(3, math.floor((mu[1] + r + 15) / 16))
    img = np.zeros((3, H, W))
    T = np.ones((H, W))
    for py in range(H):
        for px in range(W):
            inside = tx0 <= px // 16 < tx1 and ty0 <= py // 16 < ty1
            d = np.array([px, py]) - mu
            a = min(0.99, o * math.exp(-0.5 * d @ Q @ d))
            if inside and a >= 1 / 255:
                T[py, px] = 1 - a
                img[:, py, px] = a * np.array(rgb) + (1 - a) * np.array(bg)
            else:
                img[:, py, px] = bg
    np.testing.assert_allclose(out["image"], img, atol=1e-14)
    np.testing.assert_allclose(out["final_T"], T, atol=1e-15)
    assert set(np.unique(out["last_idx"])) <= {0, 1}
    assert np.array_equal(out["last_idx"] == 1, T < 1)


def test_transmittance_telescoping_identity():
    """sum_i alpha_i T_i + T_final = 1: with white Gaussians on a white
    background every pixel is exactly 1, and on black it is 1 - T_final."""
    p, view = scenes.tiny_scene(300, 64, 48, seed=7)
    p["sh"][:] = (1.0 - 0.5) / (0.5 / math.sqrt(math.pi))
    p["sh"] = p["sh"].astype(float)
    _, _, _, white = oracle.forward_view(p, view, bg=(1, 1, 1))
    np.testing.assert_allclose(white["image"], 1.0, atol=1e-12)
    _, _, _, black = oracle.forward_view(p, view, bg=(0, 0, 0))
    np.testing.assert_allclose(black["image"], np.broadcast_to(1 - black["final_T"], (3, 48, 64)),
                               atol=1e-12)
    assert (black["final_T"] < 1).mean() > 0.5


def test_early_termination_threshold():
    """Stacked opaque Gaussians: T drops by (1-alpha) per layer and the layer
    that would take T below 1e-4 is left out."""
    W, H = 16, 16
    view = scenes.camera(W, H, 16.0, 16.0, 8.0, 8.0)
    n = 6
    means = np.array([[0, 0, 1.0 + 0.1 * k] for k in range(n)])
    y00 = 0.5 / math.sqrt(math.pi)
    p = dict(means=means, log_scales=np.full((n, 3), math.log(0.5)),
             quats=np.tile([1.0, 0, 0, 0], (n, 1)), opacity_logits=np.full(n, 3.0),
             sh=np.full((1, n, 3), 0.5 / y00), sh_degree=0)
    proj, st, lst, out = oracle.forward_view(p, view)
    alpha = 1 / (1 + math.exp(-3.0)) * math.exp(-0.5 * 0 / 1)  # centre pixel (8,8), power 0
    T, k = 1.0, 0
    while k < n and T * (1 - alpha) >= 1e-4:
        T *= 1 - alpha
        k += 1
    assert out["last_idx"][8, 8] == k
    np.testing.assert_allclose(out["final_T"][8, 8], T, rtol=1e-14)
    assert out["n_eval"][8, 8] == k + 1


def test_bin_matches_lexsort():
    rng = np.random.default_rng(4)
    n, tx, ty = 500, 9, 7
    depth = rng.choice(rng.uniform(0.5, 5.0, 200), n).astype(np.float32)  # many exact ties
    x0 = rng.integers(0, tx, n)
    y0 = rng.integers(0, ty, n)
    x1 = np.minimum(tx, x0 + rng.integers(0, 4, n))
    y1 = np.minimum(ty, y0 + rng.integers(1, 4, n))
    rect = np.stack([x0, y0, x1, y1], 1).astype(np.int32)
    tt = ((x1 - x0) * (y1 - y0)).astype(np.int32)
    start, lst = oracle.bin_tiles(depth, rect, tt, tx, ty)
    tiles, dks, ids = [], [], []
    for i in range(n):
        for yy in range(y0[i], y1[i]):
            for xx in range(x0[i], x1[i]):
                tiles.append(yy * tx + xx)
                dks.append(depth[i])
                ids.append(i)
    tiles, dks, ids = np.array(tiles), np.array(dks), np.array(ids)
    order = np.lexsort((ids, dks, tiles))
    assert np.array_equal(lst, ids[order])
    assert np.array_equal(np.diff(start), np.bincount(tiles, minlength=tx * ty))


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_tiled_equals_brute_force_with_rect(tile):
    p, view = scenes.tiny_scene(64, 32, 32, seed=11)
    tw, th = tile
    proj, st, lst, out = oracle.forward_view(p, view, tw, th, bg=(0.2, 0.1, 0.0))
    bf = oracle.render_brute(proj, view, tw, th, bg=(0.2, 0.1, 0.0), use_rect=True)
    np.testing.assert_array_equal(out["image"], bf["image"])
    np.testing.assert_array_equal(out["final_T"], bf["final_T"])


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_low_opacity_is_tile_size_independent(tile):
    """The rect [floor((mu-r)/t), floor((mu+r+t-1)/t)) can stop one pixel short
    of mu + r on the high side, so a missed pixel lies more than r - 1 >= 3 sigma - 1
    from the mean.  When o exp(-(3 sigma - 1)^2 / (2 sigma^2)) < 1/255 for every
    Gaussian, no missed pixel could reach alpha = 1/255 and the tile lists change
    nothing: the tiled render equals brute force over all Gaussians, whatever the
    tile size."""
    p, view = scenes.tiny_scene(64, 32, 32, seed=12, max_opacity_logit=-3.0,
                                log_scale=(-1.5, 0.2), anisotropic=False)
    tw, th = tile
    proj, st, lst, out = oracle.forward_view(p, view, tw, th)
    vis = proj["tiles_touched"] > 0
    a, b, c = proj["cov2d"][vis].T
    sig = np.sqrt(0.5 * (a + c) + np.sqrt(0.25 * (a - c) ** 2 + b * b))
    assert np.all(proj["opacity"][vis] * np.exp(-(3 * sig - 1) ** 2 / (2 * sig ** 2)) < 1 / 255)
    bf = oracle.render_brute(proj, view, tw, th, use_rect=False)
    np.testing.assert_allclose(out["image"], bf["image"], atol=1e-15)


def test_high_opacity_depends_on_tile_size():
    """The counterpart: an opaque Gaussian whose high rect edge falls just past a
    tile boundary loses a pixel that is within alpha >= 1/255 under 8x8 tiles but
    not under 32x8 tiles, so the image depends on the tile size."""
    view = scenes.camera(64, 16, 64.0, 64.0, 0.0, 8.0)
    differs = 0
    for k in range(40):
        x = 0.35 + 0.05 * k  # sweep the mean across a few tile boundaries
        p = one_gaussian([x, 0.0, 2.0], math.log(0.06), 5.0, [1.0, 1.0, 1.0])
        a = oracle.forward_view(p, view, 8, 8)[3]["image"]
        b = oracle.forward_view(p, view, 32, 8)[3]["image"]
        differs += int(np.abs(a - b).max() > 0)
    assert differs > 0


def test_permutation_invariance():
    p, view = scenes.tiny_scene(120, 48, 40, seed=14, sh_degree=3)
    _, _, _, base = oracle.forward_view(p, view)
    perm = np.random.default_rng(1).permutation(120)
    q = scenes.subset(p, perm)
    proj, _, _, other = oracle.forward_view(q, view)
    d = proj["depth"][proj["tiles_touched"] > 0].astype(np.float32)
    assert len(np.unique(d)) == len(d)  # distinct keys: order fully fixed by depth
    np.testing.assert_array_equal(other["image"], base["image"])


def test_grayscale_is_render_of_mean_colour():
    p, view = scenes.tiny_scene(80, 40, 32, seed=15, sh_degree=0)
    gview = dict(view, channels=1)
    proj, st, lst, g = oracle.forward_view(p, gview, bg=(0.3, 0.6, 0.0))
    proj2 = dict(proj)
    proj2["rgb"] = np.repeat(proj["rgb"].mean(1, keepdims=True), 3, 1)
    rgbv = oracle.render(proj2, st, lst, view, bg=(0.3, 0.3, 0.3))
    for c in range(3):
        np.testing.assert_allclose(g["image"][0], rgbv["image"][c], atol=1e-14)


# ----------------------------------------------------------------------------
# Compositing adjoint against central differences.
# ----------------------------------------------------------------------------
def _render_scalar(proj, st, lst, view, w, bg):
    out = oracle.render(proj, st, lst, view, bg=bg)
    return float(np.sum(out["image"] * w)), out


@pytest.mark.parametrize("channels", [3, 1])
def test_render_bwd_matches_central_differences(channels):
    p, view = scenes.tiny_scene(30, 32, 24, seed=16 + channels)
    view = dict(view, channels=channels)
    bg = (0.25, 0.5, 0.75)
    proj, st, lst, _ = oracle.forward_view(p, view, bg=bg)
    rng = np.random.default_rng(2)
    w = rng.normal(size=(channels, 24, 32))
    g = oracle.render_bwd(proj, st, lst, view, w, bg=bg)
    h = 1e-6
    keys = dict(mean2d="dmean2d", conic="dconic", opacity="dopacity", rgb="drgb")
    checked = skipped = 0
    for key, gk in keys.items():
        arr = proj[key]
        flat = arr.reshape(-1)
        gflat = g[gk].reshape(-1)
        for j in range(flat.size):
            old = flat[j]
            flat[j] = old + h
            fp, op = _render_scalar(proj, st, lst, view, w, bg)
            flat[j] = old - h
            fm, om = _render_scalar(proj, st, lst, view, w, bg)
            flat[j] = old
            if not all(np.array_equal(op[k], om[k]) for k in ("last_idx", "n_eval", "n_included")):
                skipped += 1
                continue
            fd = (fp - fm) / (2 * h)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked > 0.95 * (checked + skipped)


def test_guard_attribution_closed_form():
    """A Gaussian whose alpha equals 1/255 exactly on a ring of pixels is
    named in guard_g (GPX_ALPHA), and so are those pixels in guard_px; a
    second Gaussian, with no pixel near a threshold, is not named."""
    W, H, f = 64, 48, 100.0
    view = scenes.camera(W, H, f, f, 20.0, 24.0)
    z, logit = 2.0, 0.4
    o = 1 / (1 + math.exp(-logit))
    var = 9.0 / (2.0 * math.log(255.0 * o))  # alpha(3 px from the centre) = 1/255
    s = z * math.sqrt(var - 0.3) / f
    a = one_gaussian([0.0, 0.0, z], math.log(s), logit, [0.5, 0.5, 0.5])
    b = one_gaussian([0.9307, 0.013, z + 1.0], math.log(0.01), 1.0, [0.5, 0.5, 0.5])
    p = {k: (np.concatenate([a[k], b[k]], axis=1 if k == "sh" else 0) if k != "sh_degree" else 0)
         for k in a}
    proj, st, lst, out = oracle.forward_view(p, view, 16, 16)
    assert out["guard_g"][0] & oracle.GPX_ALPHA
    assert out["guard_g"][1] == 0
    for dx, dy in ((3, 0), (-3, 0), (0, 3), (0, -3)):
        assert out["guard_px"][24 + dy, 20 + dx] & oracle.GPX_ALPHA
    # the centre pixel sits exactly on the mean: power 0, its own guard
    assert out["guard_px"][24, 20] == oracle.GPX_POWER
    assert out["guard_px"][24, 24] == 0


def test_guard_attribution_matches_pixel_bits():
    """On a random scene every guarded pixel has, among the list entries it
    examined, a Gaussian whose own decision there is in the guard band
    (alpha within 5e-5 relative of 1/255, recomputed here), and that
    Gaussian is named in guard_g; guard_g names no Gaussian for a bit that
    no pixel carries."""
    p, view = scenes.tiny_scene(3000, 128, 96, seed=8)
    proj, st, lst, out = oracle.forward_view(p, view, 8, 8)
    gpx, gg = out["guard_px"], out["guard_g"]
    assert np.bitwise_or.reduce(gg.ravel()) == np.bitwise_or.reduce(gpx.ravel())
    tx = (view["width"] + 7) // 8
    ys, xs = np.nonzero(gpx & oracle.GPX_ALPHA)
    assert len(ys) > 0
    for py, px in zip(ys, xs):
        t = (py // 8) * tx + px // 8
        ids = lst[st[t]:st[t + 1]][: out["n_eval"][py, px]]
        dx, dy = proj["mean2d"][ids, 0] - px, proj["mean2d"][ids, 1] - py
        a, b, c = proj["conic"][ids].T
        oG = proj["opacity"][ids] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
        near = np.abs(oG * 255.0 - 1.0) < 5e-5
        assert near.any(), (py, px)
        assert np.all(gg[ids[near]] & oracle.GPX_ALPHA)

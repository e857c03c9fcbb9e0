"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the
same seeded inputs.

Bars (stated against the FP64 oracle):
  * tile rects, tiles touched, radii, FP32 depth keys, tile lists and their
    order: bit-exact (outside the oracle's guard bands, which are counted);
  * images and final transmittance: max-abs <= 1e-5 on every pixel outside
    the guard bands; last_idx exact there;
  * gradients: relative L2 <= 1e-4 per parameter group;
  * loss: relative 1e-5; Adam: relative 1e-6 per element.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2409_13055_gb300 import binding as B
from paper_2409_13055_gb300 import mapping, scenes
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_13055_gb300 import build
    build.build()
    B.lib()


def posed(view, seed, trans=0.3, ang=20.0):
    R, t = scenes.random_pose(np.random.default_rng(seed), trans, ang)
    return dict(view, R=R, t=t * 0.3)


CASES = {
    "planes10k": lambda: (scenes.planes_scene(), scenes.camera(320, 240, 300.0, 300.0, 160.0, 120.0)),
    "tiny_sh3_posed": lambda: (lambda p_v: (p_v[0], posed(p_v[1], 5)))(
        scenes.tiny_scene(600, 96, 72, seed=21, sh_degree=3)),
    "tiny_sh2_posed": lambda: (lambda p_v: (p_v[0], posed(p_v[1], 6)))(
        scenes.tiny_scene(500, 80, 64, seed=22, sh_degree=2)),
    "room20k_sh3": lambda: (scenes.room_scene(20_000, seed=31), scenes.camera(160, 120, 131.25, 131.25)),
}


def run_forward(p, view, tile=(16, 16), batch=128, bg=(0.0, 0.0, 0.0)):
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 21, tile=tile,
                              smem_batch=batch, bg=bg)
    rast.forward(gm.gs_map())
    torch.cuda.synchronize()
    return gm, rast


@pytest.mark.parametrize("case", list(CASES))
def test_projection_parity(case):
    p, view = CASES[case]()
    gm, rast = run_forward(p, view)
    g = U.gpu_projection(rast, gm.n)
    o = oracle.project(p, view)
    guard = (o["guard"] & U.FWD_GUARDS) != 0
    assert guard.sum() <= max(1, 1e-3 * guard.size), guard.sum()  # one of a few hundred may be
    ok = ~guard
    vis = o["tiles_touched"] > 0
    assert vis.sum() > 50
    np.testing.assert_array_equal(g["touched"][ok], o["tiles_touched"][ok])
    np.testing.assert_array_equal(g["radius"][ok & vis], o["radius"][ok & vis])
    np.testing.assert_array_equal(g["rect"][ok & vis], o["rect"][ok & vis])
    m = ok & vis
    # depth key: the correctly rounded FP32 depth
    np.testing.assert_array_equal(g["depth32"][m], o["depth"][m].astype(np.float32))
    np.testing.assert_allclose(g["mean2d"][m], o["mean2d"][m], rtol=0, atol=1e-7)
    cn = np.linalg.norm(o["conic"][m], axis=1, keepdims=True)
    assert np.max(np.abs(g["conic"][m] - o["conic"][m]) / cn) < 2e-5
    np.testing.assert_allclose(g["opacity"][m], o["opacity"][m], rtol=1e-6, atol=0)
    np.testing.assert_allclose(g["rgb"][m], o["rgb"][m], rtol=0, atol=2e-6)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_binning_bit_exact(case, tile):
    p, view = CASES[case]()
    gm, rast = run_forward(p, view, tile=tile)
    g = U.gpu_projection(rast, gm.n)
    ranges, keys, vals, c = U.gpu_tile_lists(rast)
    assert c.status == 0 and c.n_instances == c.n_instances_raw
    tx, ty = oracle.tile_grid(view["width"], view["height"], *tile)
    # 1. the integer part alone: the GPU's own (tile, Gaussian) pairs, each
    #    Gaussian with as many as it counted, inside its rect, and in the
    #    (tile, FP32 depth key, index) order
    np.testing.assert_array_equal(np.bincount(vals, minlength=gm.n), g["touched"])
    r = g["rect"][vals]
    kx, ky = keys % tx, keys // tx
    assert np.all((kx >= r[:, 0]) & (kx < r[:, 2]) & (ky >= r[:, 1]) & (ky < r[:, 3]))
    order = np.lexsort((vals, g["depth32"][vals], keys))
    np.testing.assert_array_equal(order, np.arange(len(vals)))
    start = np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=tx * ty))])
    np.testing.assert_array_equal(ranges[:, 0], start[:-1])
    np.testing.assert_array_equal(ranges[:, 1], start[1:])
    assert len(np.unique(keys.astype(np.int64) * gm.n + vals)) == len(vals)  # no pair twice
    # 2. end to end: lists from the oracle's own projection and binning, the
    #    Gaussians with a guarded projection decision removed from both sides
    o = oracle.project(p, view, *tile)
    compared, removed = U.compare_tile_lists(keys, vals, gm.n, o, view, tile)
    print(f"{case} {tile}: {compared} pairs bit-exact, {removed} of guarded Gaussians removed")
    assert compared > 100 and removed <= max(50, 0.01 * compared)


def test_emission_of_large_gaussians_in_several_rounds():
    """Gaussians that cover the whole image (768 tiles each, taller than the
    16 stored span rows, so their rows come from the span pool) among small
    ones: an emission CTA's entries then hold ~10k instances, written in
    several rounds of per-thread runs.  The lists are checked as in
    test_binning_bit_exact, against the GPU's own counts and the oracle."""
    tile = (8, 8)
    p, view = scenes.tiny_scene(400, 256, 192, seed=41, sh_degree=1)
    big = np.arange(0, 400, 13)  # 31 Gaussians
    p["log_scales"][big] = np.log(1.5)
    p["opacity_logits"][big] = 3.0
    gm, rast = run_forward(p, view, tile=tile)
    g = U.gpu_projection(rast, gm.n)
    ranges, keys, vals, c = U.gpu_tile_lists(rast)
    assert c.status == 0 and c.n_instances == c.n_instances_raw
    tx, ty = oracle.tile_grid(view["width"], view["height"], *tile)
    assert np.sum(g["touched"][big] == tx * ty) >= 10  # whole-image boxes
    assert c.n_instances > 2 * 2048
    np.testing.assert_array_equal(np.bincount(vals, minlength=gm.n), g["touched"])
    order = np.lexsort((vals, g["depth32"][vals], keys))
    np.testing.assert_array_equal(order, np.arange(len(vals)))
    start = np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=tx * ty))])
    np.testing.assert_array_equal(ranges[:, 0], start[:-1])
    np.testing.assert_array_equal(ranges[:, 1], start[1:])
    o = oracle.project(p, view, *tile)
    compared, removed = U.compare_tile_lists(keys, vals, gm.n, o, view, tile)
    # a whole-image box meets many tile edges, so a few of them are guarded
    # (6 of the 400 Gaussians here, 3844 of 28156 pairs)
    assert compared > 20000 and np.count_nonzero(o["guard"]) <= 10


def test_depth_order_holds_the_visible_pairs_and_binning_repeats():
    """The first depth pass drops the culled pairs: the depth order lists
    exactly the Gaussians with a tile, by (FP32 depth key, index), and a
    second binning of the same projection yields the same tile lists."""
    p, view = CASES["room20k_sh3"]()
    gm, rast = run_forward(p, view)
    g = U.gpu_projection(rast, gm.n)
    vis = np.nonzero(g["touched"] > 0)[0]
    assert 0 < len(vis) < gm.n
    order = rast.buffer(B.GS_BUF_DEPTH_ORDER, torch.int32)[: len(vis)].cpu().numpy()
    np.testing.assert_array_equal(order, vis[np.lexsort((vis, g["depth32"][vis]))])
    first = U.gpu_tile_lists(rast)
    rast.bin_sort(gm.n)
    torch.cuda.synchronize()
    second = U.gpu_tile_lists(rast)
    assert second[3].status == 0
    for a, b in zip(first[:3], second[:3]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("case", list(CASES))
def test_tight_rects_same_render_fewer_instances(case):
    """Square against tight tile rects on the GPU: the tight lists are
    shorter, while the image, the final transmittance and the loss are bit-
    identical and the parameter gradients equal up to the order of float
    atomics; the square rects match the oracle's square rects."""
    p, view = CASES[case]()
    target = scenes.random_target(view, 3)
    out = {}
    for tight in (False, True):
        gm = mapping.GaussianMap(p)
        rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 21, tight_rect=tight,
                                  bg=(0.1, 0.2, 0.3))
        rast.forward(gm.gs_map())
        rast.loss_l1_ssim(rast.pack([target]), 0.2)
        rast.render_bwd(gm.gs_map(), gm.gs_map_grad())
        torch.cuda.synchronize()
        c = rast.counters()
        assert c.status == 0
        out[tight] = dict(img=rast.images.clone(), T=rast.final_T.clone(),
                          grad=gm.grad.clone().cpu().numpy(), n=int(c.n_instances),
                          proj=U.gpu_projection(rast, gm.n), loss=rast.loss.item())
    sq, ti = out[False], out[True]
    assert ti["n"] < sq["n"]
    assert torch.equal(sq["img"], ti["img"]) and torch.equal(sq["T"], ti["T"])
    assert sq["loss"] == ti["loss"]
    assert U.rel_l2(ti["grad"], sq["grad"]) < 1e-5
    o = oracle.project(p, view, tight=False)
    ok = ((o["guard"] & U.FWD_GUARDS) == 0) & (o["tiles_touched"] > 0)
    np.testing.assert_array_equal(sq["proj"]["rect"][ok], o["rect"][ok])
    np.testing.assert_array_equal(sq["proj"]["touched"][ok], o["tiles_touched"][ok])


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_render_parity(case, tile):
    p, view = CASES[case]()
    bg = (0.1, 0.2, 0.3)
    gm, rast = run_forward(p, view, tile=tile, bg=bg)
    img = rast.view_slice(rast.images, 0).cpu().numpy()
    T = rast.view_slice(rast.final_T, 0, per_pixel=True).cpu().numpy()
    last = rast.view_slice(rast.last_idx, 0, per_pixel=True).cpu().numpy()
    proj, st, lst, o = oracle.forward_view(p, view, tile[0], tile[1], bg)
    mask = U.guard_pixel_mask(view, proj, o, tile)
    assert mask.mean() < 0.02, mask.mean()
    ok = ~mask
    err = np.abs(img - o["image"])[:, ok]
    assert err.max() <= IMG_TOL, (err.max(), np.unravel_index(np.argmax(np.abs(img - o["image"]) * ok), img.shape))
    assert np.abs(T - o["final_T"])[ok].max() <= IMG_TOL
    np.testing.assert_array_equal(last[ok], o["last_idx"][ok])


@pytest.mark.parametrize("tile,ppts", [((16, 16), (1, 2, 4, 8)), ((8, 8), (1, 2)),
                                       ((32, 8), (1, 2, 4, 8))])
def test_pixels_per_thread_do_not_change_results(tile, ppts):
    """Register blocking changes only which thread evaluates a pixel: images,
    transmittance and last_idx are bit-identical for every pixels_per_thread,
    and gradients agree up to the order of the float atomics."""
    p, view = CASES["tiny_sh3_posed"]()
    target = scenes.random_target(view, 31)
    ref = None
    for ppt in ppts:
        gm = mapping.GaussianMap(p)
        rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 18, tile=tile,
                                  pixels_per_thread=ppt, bg=(0.1, 0.2, 0.3))
        m, g = gm.gs_map(), gm.gs_map_grad()
        rast.forward(m)
        rast.loss_l1_ssim(rast.pack([target]), 0.2)
        rast.render_bwd(m, g)
        torch.cuda.synchronize()
        out = (rast.images.clone(), rast.final_T.clone(), rast.last_idx.clone(), gm.grad.clone())
        if ref is None:
            ref = out
            continue
        assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
        assert torch.equal(out[2], ref[2])
        assert U.rel_l2(out[3].cpu().numpy(), ref[3].cpu().numpy()) < 1e-5


@pytest.mark.parametrize("tile,ppt", [((16, 16), 1), ((8, 8), 2)])
def test_render_grayscale_and_mixed_batch(tile, ppt):
    """One launch over three views of different sizes and channel counts equals
    the oracle view by view, with one tile per CTA and with one tile per warp
    (8x8 tiles at two pixels per thread, where one CTA holds tiles of
    different views)."""
    p = scenes.room_scene(20_000, seed=41)
    views = [scenes.camera(160, 120, 131.25, 131.25),
             dict(scenes.camera(188, 120, 115.0, 115.0, channels=1)),
             posed(scenes.camera(300, 170, 150.0, 150.0), 7, 0.2, 10.0)]
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer(views, gm.n, instance_capacity=1 << 21, bg=(0.2, 0.4, 0.6),
                              tile=tile, pixels_per_thread=ppt)
    rast.forward(gm.gs_map())
    torch.cuda.synchronize()
    for v, view in enumerate(views):
        img = rast.view_slice(rast.images, v).cpu().numpy()
        proj, st, lst, o = oracle.forward_view(p, view, tile[0], tile[1], bg=(0.2, 0.4, 0.6))
        ok = ~U.guard_pixel_mask(view, proj, o, tile)
        assert np.abs(img - o["image"])[:, ok].max() <= IMG_TOL


def test_maximum_view_count_batch():
    """GS_MAX_VIEWS views of two ragged sizes and both channel counts in one
    plan: sampled views equal the oracle's render, and the batch loss is the
    mean of the oracle's per-view losses of the rendered images."""
    p = scenes.room_scene(5_000, seed=51)
    views = []
    for i in range(B.GS_MAX_VIEWS):
        w, h = (40, 30) if i % 2 == 0 else (26, 18)
        views.append(posed(scenes.camera(w, h, 30.0, 30.0, channels=1 if i % 3 == 0 else 3),
                           100 + i, 0.1, 5.0))
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer(views, gm.n, instance_capacity=1 << 20, bg=(0.1, 0.2, 0.3))
    rast.forward(gm.gs_map())
    targets = [scenes.random_target(v, 200 + i) for i, v in enumerate(views)]
    rast.loss_l1_ssim(rast.pack(targets), 0.2)
    torch.cuda.synchronize()
    assert rast.counters().status == 0
    imgs = [rast.view_slice(rast.images, v).cpu().numpy() for v in range(len(views))]
    for v in (0, 1, 3, 32, 62, 63):
        proj, st, lst, o = oracle.forward_view(p, views[v], 16, 16, bg=(0.1, 0.2, 0.3))
        ok = ~U.guard_pixel_mask(views[v], proj, o, (16, 16))
        assert ok.mean() > 0.5
        assert np.abs(imgs[v] - o["image"])[:, ok].max() <= IMG_TOL, v
    L = np.mean([oracle.loss_l1_ssim(im.astype(np.float64), t.astype(np.float64), 0.2,
                                     want_grad=False)[0] for im, t in zip(imgs, targets)])
    assert abs(rast.loss.item() - L) <= 1e-5 * abs(L)


def test_order_invariance_bit_identical():
    """Permuting the input Gaussians leaves the image bit-identical.  Ties of
    the FP32 depth key are broken by index, so the permutation keeps tied
    Gaussians in their original relative order (the oracle's keys decide the
    ties)."""
    p = scenes.room_scene(20_000, seed=31)
    view = posed(scenes.camera(160, 120, 131.25, 131.25), 11, 0.2, 10.0)
    n = p["means"].shape[0]
    key = oracle.project(p, view)["depth"].astype(np.float32)
    perm = np.random.default_rng(3).permutation(n)
    # restore the original order inside every group of equal keys
    by_key = {}
    for pos, g in enumerate(perm):
        by_key.setdefault(key[g], []).append(pos)
    for k, positions in by_key.items():
        if len(positions) > 1:
            perm[positions] = np.sort(perm[positions])
    _, r1 = run_forward(p, view)
    _, r2 = run_forward(scenes.subset(p, perm), view)
    assert torch.equal(r1.images, r2.images)
    assert torch.equal(r1.final_T, r2.final_T)


def test_empty_and_degenerate():
    # no Gaussian in front of the camera: background everywhere
    p = scenes.tiny_scene(50, 40, 30, seed=3)[0]
    p["means"][:, 2] = -1.0
    view = scenes.camera(40, 30, 40.0, 40.0)
    gm, rast = run_forward(p, view, bg=(0.25, 0.5, 0.75))
    img = rast.view_slice(rast.images, 0).cpu().numpy()
    np.testing.assert_array_equal(img, np.broadcast_to(np.array([0.25, 0.5, 0.75], np.float32)[:, None, None], img.shape))
    assert torch.all(rast.final_T == 1) and torch.all(rast.last_idx == 0)
    assert rast.counters().n_instances == 0
    # one Gaussian, a 1x1 image and a ragged 17x9 image
    for (w, h) in [(1, 1), (17, 9)]:
        p = scenes.tiny_scene(1, w, h, seed=4)[0]
        p["means"][0] = [0.0, 0.0, 1.0]
        view = scenes.camera(w, h, float(w), float(w))
        gm, rast = run_forward(p, view)
        proj, st, lst, o = oracle.forward_view(p, view)
        np.testing.assert_allclose(rast.view_slice(rast.images, 0).cpu().numpy(), o["image"],
                                   atol=IMG_TOL)


def test_capacity_overflow_sets_status():
    p, view = CASES["planes10k"]()
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer([view], gm.n, instance_capacity=1000)
    rast.forward(gm.gs_map())
    c = rast.counters()
    assert c.status & B.GS_DEV_CAPACITY
    assert c.n_instances == 1000 and c.n_instances_raw > 1000


def test_nonfinite_gaussian_is_culled_and_flagged():
    p, view = CASES["tiny_sh3_posed"]()
    p["means"][3, 0] = np.nan
    p["log_scales"][7, 1] = np.inf
    gm, rast = run_forward(p, view)
    c = rast.counters()
    assert c.status & B.GS_DEV_NONFINITE
    g = U.gpu_projection(rast, gm.n)
    assert g["touched"][3] == 0 and g["touched"][7] == 0
    assert torch.isfinite(rast.images).all()


# ----------------------------------------------------------------------------
# Loss, backward, Adam.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
@pytest.mark.parametrize("shape", [(3, 48, 80), (1, 37, 53)])
def test_loss_parity(lam, shape):
    rng = np.random.default_rng(5)
    C, H, W = shape
    view = scenes.camera(W, H, float(W), float(W), channels=C)
    img = rng.uniform(0, 1, shape).astype(np.float32)
    tgt = rng.uniform(0, 1, shape).astype(np.float32)
    rast = mapping.Rasterizer([view], 16, instance_capacity=1024)
    ti, tt = rast.pack([img]), rast.pack([tgt])
    rast.loss_l1_ssim(tt, lam, images=ti)
    torch.cuda.synchronize()
    L, d = oracle.loss_l1_ssim(img, tgt, lam)
    assert abs(rast.loss.item() - L) <= 1e-5 * max(1.0, abs(L))
    gd = rast.view_slice(rast.dL, 0).cpu().numpy()
    assert U.rel_l2(gd, d) < 1e-5
    assert np.abs(gd - d).max() <= 1e-5 * np.abs(d).max()


def backward_case(p, view, lam, tile=(16, 16)):
    bg = (0.1, 0.2, 0.3)
    target = scenes.random_target(view, 17)
    proj, st, lst, o = oracle.forward_view(p, view, tile[0], tile[1], bg)
    L, dimg = oracle.loss_l1_ssim(o["image"], target, lam)
    mask = U.guard_pixel_mask(view, proj, o, tile) | U.grad_pixel_mask(o)
    dimg = dimg * (~mask)[None]
    og = oracle.project_bwd(p, view, oracle.render_bwd(proj, st, lst, view, dimg, tile[0], tile[1], bg),
                            tile_w=tile[0], tile_h=tile[1])
    gm, rast = run_forward(p, view, tile=tile, bg=bg)
    dL = rast.pack([dimg])
    rast.render_bwd(gm.gs_map(), gm.gs_map_grad(), dL=dL)
    torch.cuda.synchronize()
    gg = {k: v.cpu().numpy() for k, v in gm.grads().items()}
    kink = (proj["guard"] & oracle.GUARD_KINK) != 0
    return og, gg, kink


@pytest.mark.parametrize("case", list(CASES))
def test_backward_parity(case):
    p, view = CASES[case]()
    og, gg, kink = backward_case(p, view, 0.2)
    assert kink.mean() < 1e-3
    for k in og:
        a, b = gg[k], og[k]
        if k == "sh":
            a, b = a[:, ~kink], b[:, ~kink]
        else:
            a, b = a[~kink], b[~kink]
        if np.linalg.norm(b) == 0:
            assert np.linalg.norm(a) < 1e-20, k
            continue
        assert U.rel_l2(a, b) <= GRAD_TOL, (k, U.rel_l2(a, b))


def test_split_backward_equals_combined():
    """gs_render_bwd_pixels followed by gs_project_bwd equals gs_render_bwd
    (up to the order of the float atomics), and accumulate = 1 adds."""
    p, view = CASES["tiny_sh3_posed"]()
    target = scenes.random_target(view, 41)
    out = []
    for split in (False, True):
        gm = mapping.GaussianMap(p)
        rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 18)
        m, g = gm.gs_map(), gm.gs_map_grad()
        rast.forward(m)
        rast.loss_l1_ssim(rast.pack([target]), 0.2)
        if split:
            rast.render_bwd_pixels()
            rast.project_bwd(m, g, accumulate=False)
        else:
            rast.render_bwd(m, g)
        torch.cuda.synchronize()
        out.append(gm.grad.clone().cpu().numpy())
        if split:
            rast.project_bwd(m, g, accumulate=True)
            torch.cuda.synchronize()
            twice = gm.grad.clone().cpu().numpy()
    assert U.rel_l2(out[1], out[0]) < 1e-5
    assert U.rel_l2(twice, 2.0 * out[1]) < 1e-6


FUSED_CASES = {
    # 600 Gaussians: four full chunks of the fused kernel and a ragged one
    "tiny_sh3_posed": lambda: (CASES["tiny_sh3_posed"]()[0], [CASES["tiny_sh3_posed"]()[1]]),
    # SH degree 0, 10k Gaussians
    "planes10k": lambda: (CASES["planes10k"]()[0], [CASES["planes10k"]()[1]]),
    # three views of different sizes, one grayscale: gradients summed over views
    "room20k_three_views": lambda: (scenes.room_scene(20_000, seed=41), [
        scenes.camera(160, 120, 131.25, 131.25),
        dict(scenes.camera(188, 120, 115.0, 115.0, channels=1)),
        posed(scenes.camera(300, 170, 150.0, 150.0), 7, 0.2, 10.0)]),
}


@pytest.mark.parametrize("case", list(FUSED_CASES))
def test_fused_projection_adjoint_adam_is_bit_identical(case):
    """gs_project_bwd_adam equals gs_project_bwd into a zeroed gradient followed
    by gs_adam_step, bit for bit, from the same screen-space gradients; with
    grads_acc it adds the given gradients first."""
    p, views = FUSED_CASES[case]()
    targets = [scenes.random_target(v, 51 + i) for i, v in enumerate(views)]
    g1, g2 = mapping.GaussianMap(p), mapping.GaussianMap(p)
    for gm in (g1, g2):  # non-trivial moments and step count
        gm.m.normal_(0, 1e-3)
        gm.v.uniform_(0, 1e-6)
        gm.step.fill_(3)
    g2.m.copy_(g1.m)
    g2.v.copy_(g1.v)
    rast = mapping.Rasterizer(views, g1.n, instance_capacity=1 << 21)
    rast.forward(g1.gs_map())
    rast.loss_l1_ssim(rast.pack(targets), 0.2)
    rast.render_bwd_pixels()
    rast.project_bwd(g1.gs_map(), g1.gs_map_grad())
    g1.adam_step()
    g2.grad.fill_(7.0)
    rast.project_bwd_adam(g2, grads_out=g2.gs_map_grad())
    torch.cuda.synchronize()
    assert g1.step.item() == g2.step.item() == 4
    groups = lambda gm, buf: torch.cat([t.reshape(-1) for t in gm._views(buf).values()])
    assert groups(g1, g1.grad).abs().sum() > 0
    for a, b in ((g1.grad, g2.grad), (g1.data, g2.data), (g1.m, g2.m), (g1.v, g2.v)):
        assert torch.equal(groups(g1, a), groups(g2, b))
    # accumulation: grads_acc = the same gradient again doubles it
    acc = mapping.GaussianMap(p)
    acc.grad.copy_(g1.grad)
    g3 = mapping.GaussianMap(p)
    rast.project_bwd_adam(g3, grads_acc=acc.gs_map_grad(), grads_out=g3.gs_map_grad())
    torch.cuda.synchronize()
    torch.testing.assert_close(groups(g3, g3.grad), 2.0 * groups(g1, g1.grad), rtol=1e-6, atol=0)


def test_adam_parity():
    rng = np.random.default_rng(8)
    n = 100_003  # ragged: not a multiple of the float4 width
    p0 = rng.normal(size=n)
    t = torch.tensor(p0, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(t)
    v = torch.zeros_like(t)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    offs = [0, 40_000, 70_001, n]
    lrs = [1e-3, 5e-2, 3e-4]
    po, mo, vo = p0.astype(np.float32).astype(np.float64), np.zeros(n), np.zeros(n)
    for s in range(1, 4):
        g = rng.normal(size=n).astype(np.float32)
        B.gs_adam_step(t, torch.from_numpy(g).cuda(), m, v, offs, lrs, 0.9, 0.999, 1e-15, step)
        for k in range(3):
            sl = slice(offs[k], offs[k + 1])
            pp, mm, vv = po[sl].copy(), mo[sl].copy(), vo[sl].copy()
            oracle.adam(pp, g[sl].astype(np.float64), mm, vv, lrs[k], s)
            po[sl], mo[sl], vo[sl] = pp, mm, vv
    torch.cuda.synchronize()
    assert step.item() == 3
    np.testing.assert_allclose(t.cpu().numpy(), po, rtol=1e-6, atol=1e-6 * 5e-2)
    np.testing.assert_allclose(m.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)


def test_full_iteration_matches_oracle():
    """Config-1 shaped iteration (10k Gaussians on planes, 320x240, L1):
    loss and every gradient group against the oracle's whole iteration."""
    p, v, targets, lam = scenes.workload("planes10k_320x240")
    view = v[0]
    L, og, renders = oracle.iteration(p, v, targets, lam)
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer(v, gm.n, instance_capacity=1 << 20)
    step = mapping.MappingStep(gm, rast, rast.pack(targets), lam)
    m, g = gm.gs_map(), gm.gs_map_grad()
    rast.forward(m)
    rast.loss_l1_ssim(step.targets, lam)
    rast.render_bwd(m, g)
    torch.cuda.synchronize()
    assert abs(rast.loss.item() - L) < 1e-5
    mask = U.guard_pixel_mask(view, oracle.project(p, view), renders[0])
    assert mask.mean() < 0.02
    gg = {k: t.cpu().numpy() for k, t in gm.grads().items()}
    keep = U.gradient_keep(p, v, renders)
    assert keep.mean() > 0.97, keep.mean()
    og = {k: g for k, g in og.items() if np.linalg.norm(g) > 0}  # identity rotations, SH-0
    errs = U.grad_errors(gg, og, keep)
    assert all(e <= GRAD_TOL for e in errs.values()), errs


def test_recompute_is_bit_identical():
    """Re-running projection and binning reproduces every workspace buffer
    bit for bit (the recompute mode relies on it)."""
    p, view = CASES["room20k_sh3"]()
    gm, rast = run_forward(p, view)
    bufs = [B.GS_BUF_PROJ, B.GS_BUF_RECT, B.GS_BUF_TOUCHED, B.GS_BUF_DEPTH_ORDER,
            B.GS_BUF_TILE_KEYS, B.GS_BUF_TILE_VALUES, B.GS_BUF_RANGES]
    I = rast.counters().n_instances
    snap = [rast.buffer(b).clone() for b in bufs]
    rast.ws[rast.buffer(B.GS_BUF_PROJ).data_ptr() - rast.ws.data_ptr():].zero_()
    rast.project(gm.gs_map())
    rast.bin_sort(gm.n)
    torch.cuda.synchronize()
    # the depth order is defined on its first entries, one per visible pair
    n_vis = int((rast.buffer(B.GS_BUF_TOUCHED, torch.int32) != 0).sum().item())
    assert 0 < n_vis < gm.n
    for b, s in zip(bufs, snap):
        cur = rast.buffer(b)
        if b in (B.GS_BUF_TILE_KEYS, B.GS_BUF_TILE_VALUES):
            assert torch.equal(cur[: 4 * I], s[: 4 * I])
        elif b == B.GS_BUF_DEPTH_ORDER:
            assert torch.equal(cur[: 4 * n_vis], s[: 4 * n_vis])
        else:
            assert torch.equal(cur, s), b


def test_autograd_function_and_recompute_mode():
    p, view = CASES["tiny_sh3_posed"]()
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 18)
    P = gm.params()
    target = torch.from_numpy(scenes.random_target(view, 3)).cuda().reshape(-1)
    grads = []
    for recompute in (False, True):
        leaves = [P[k].detach().clone().contiguous().requires_grad_(True)
                  for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
        img = mapping.GSRender.apply(*leaves, rast, recompute)
        loss = (img - target).abs().mean()
        loss.backward()
        grads.append([l.grad.clone() for l in leaves])
    for a, b in zip(*grads):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-9)
    # against the oracle: L1 loss gradient through the same path
    o_L, og, renders = oracle.iteration(
        p, [view], [target.view(3, view["height"], view["width"]).cpu().numpy()], 0.0)
    keep = U.gradient_keep(p, [view], renders)
    assert keep.mean() > 0.95, keep.mean()
    got = dict(zip(("means", "log_scales", "quats", "opacity_logits", "sh"),
                   (g.cpu().numpy() for g in grads[0])))
    errs = U.grad_errors(got, og, keep)
    assert all(e <= GRAD_TOL for e in errs.values()), errs


@pytest.mark.parametrize("sh_degree", [3, 1])
def test_grouped_adjoint_and_adam_are_bit_identical(sh_degree):
    """Without keep_grads, MappingStep neither writes nor reads the gradient
    of groups of 32 Gaussians that touch no tile: the parameters and moments
    after three iterations equal the dense path's bit for bit (deterministic
    adjoint, so both see the same gradients), with both kinds of group
    present (the map in Z-order, so a view's invisible Gaussians cluster)."""
    p, view = CASES["room20k_sh3"]()
    p = scenes.z_ordered(p)
    if sh_degree != 3:
        K = (sh_degree + 1) ** 2
        p = dict(p, sh=np.ascontiguousarray(p["sh"][:K]), sh_degree=sh_degree)  # [K, n, 3]
    target = scenes.random_target(view, 77)
    out = []
    for keep in (True, False):
        gm = mapping.GaussianMap(p)
        rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 20, tile=(8, 8),
                                  pixels_per_thread_bwd=2, deterministic=True)
        step = mapping.MappingStep(gm, rast, rast.pack([target]), 0.2, keep_grads=keep)
        assert step.groups == (not keep)
        for _ in range(3):
            step.run()
        torch.cuda.synchronize()
        out.append((gm.data.clone(), gm.m.clone(), gm.v.clone(), gm.step.item()))
        if not keep:
            gv = step.group_vis.cpu().numpy()
            assert gv.min() == 0 and gv.max() == 1, np.bincount(gv)
    assert out[0][3] == out[1][3] == 3
    for a, b in zip(out[0][:3], out[1][:3]):
        assert torch.equal(a, b)


def test_host_pipeline_matches_direct_steps():
    """HostPipeline (inputs copied from pinned host memory on a copy stream,
    loss read back one iteration late) gives the losses and updates of
    eager iterations on device-resident inputs, with a different target and
    pose each iteration."""
    p, view = CASES["tiny_sh3_posed"]()
    views = [posed(view, 30 + i, 0.05, 3.0) for i in range(4)]
    targets = [scenes.random_target(view, 40 + i) for i in range(4)]
    # direct: eager iterations, inputs written on the device
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer([views[0]], gm.n, instance_capacity=1 << 18)
    step = mapping.MappingStep(gm, rast, rast.pack([targets[0]]), 0.2)
    start = gm.data.clone()
    want = []
    for v, t in zip(views, targets):
        rast.views_dev.copy_(mapping.views_to_device([v], rast.device)[1])
        step.targets.copy_(rast.pack([t]))
        step.run()
        want.append(rast.loss.item())
    want_delta = (gm.data - start).cpu().numpy()
    # pipelined, from pinned host buffers
    gm2 = mapping.GaussianMap(p)
    rast2 = mapping.Rasterizer([views[0]], gm2.n, instance_capacity=1 << 18)
    step2 = mapping.MappingStep(gm2, rast2, rast2.pack([targets[0]]), 0.2)
    snapshot = (gm2.data.clone(), gm2.m.clone(), gm2.v.clone(), gm2.step.clone())
    pipe = mapping.HostPipeline(step2, warmup=1)
    for buf, val in zip((gm2.data, gm2.m, gm2.v, gm2.step), snapshot):
        buf.copy_(val)  # undo the capture's warm-up iteration
    got = []
    for v, t in zip(views, targets):
        hv = mapping.views_to_device([v], "cpu")[1].pin_memory()
        ht = torch.as_tensor(np.ascontiguousarray(t, np.float32)).reshape(-1).pin_memory()
        prev = pipe.submit(ht, hv)
        if prev is not None:
            got.append(prev)
    got.append(pipe.drain())
    torch.cuda.synchronize()
    assert len(got) == 4
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=0)
    assert U.rel_l2((gm2.data - snapshot[0]).cpu().numpy(), want_delta) < 1e-3


def test_cuda_graph_replay_matches_eager():
    """Three iterations replayed from one captured CUDA graph equal three eager
    iterations: same step counter, same gradients of the last iteration and
    the same parameter updates (up to the order of the backward's float
    atomics)."""
    p, view = CASES["tiny_sh3_posed"]()
    target = scenes.random_target(view, 12)
    runs = []
    for use_graph in (False, True):
        gm = mapping.GaussianMap(p)
        rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 18)
        step = mapping.MappingStep(gm, rast, rast.pack([target]), 0.2, keep_grads=True)
        if use_graph:
            step.capture(warmup=0)
        start = gm.data.clone()
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        runs.append((gm.data - start, gm.grad.clone(), gm.step.item()))
    assert runs[0][2] == runs[1][2] == 3
    assert U.rel_l2(runs[1][1].cpu().numpy(), runs[0][1].cpu().numpy()) < 1e-5
    assert U.rel_l2(runs[1][0].cpu().numpy(), runs[0][0].cpu().numpy()) < 1e-3


def test_batched_equals_per_view_loop():
    """One batched launch over three mixed views and the loop of three
    single-view plans compute the same loss and gradients (up to the order of
    the backward's float atomics)."""
    p = scenes.room_scene(30_000, seed=51)
    views = [scenes.camera(160, 120, 131.25, 131.25),
             posed(scenes.camera(188, 120, 115.0, 115.0, channels=1), 8, 0.2, 10.0),
             posed(scenes.camera(200, 112, 100.0, 100.0), 9, 0.2, 10.0)]
    targets = [scenes.random_target(v, 60 + i) for i, v in enumerate(views)]
    out = []
    for batched in (True, False):
        gm = mapping.GaussianMap(p)
        if batched:
            rast = mapping.fit_instance_capacity(views, gm)
            it = mapping.MappingStep(gm, rast, rast.pack(targets), 0.2, keep_grads=True)
            loss = lambda: rast.loss.item()
        else:
            it = mapping.PerViewLoop(gm, views, targets, 0.2, keep_grads=True)
            loss = lambda: sum(r.loss.item() for r in it.rasts)
        it()
        torch.cuda.synchronize()
        out.append((gm.grad.clone().cpu().numpy(), loss()))
    assert abs(out[0][1] - out[1][1]) < 1e-6
    assert U.rel_l2(out[0][0], out[1][0]) < 1e-5


def test_long_tile_lists():
    """12000 small Gaussians crowded in front of a 64x48 view give tiles of
    up to ~10k entries: the lists equal the oracle's, and the image too."""
    rng = np.random.default_rng(77)
    n = 12000
    view = scenes.camera(64, 48, 64.0, 64.0)
    z = rng.uniform(1.0, 3.0, n)
    u, v = rng.uniform(24, 40, n), rng.uniform(16, 32, n)
    q = rng.normal(size=(n, 4))
    p = dict(means=np.stack([(u - 32) / 64 * z, (v - 24) / 64 * z, z], 1).astype(np.float32),
             log_scales=np.full((n, 3), -2.5, np.float32) + rng.normal(0, 0.2, (n, 3)).astype(np.float32),
             quats=(q / np.linalg.norm(q, axis=1)[:, None]).astype(np.float32),
             opacity_logits=rng.normal(-3.0, 0.5, n).astype(np.float32),
             sh=rng.normal(0, 0.3, (1, n, 3)).astype(np.float32), sh_degree=0)
    gm, rast = run_forward(p, view, tile=(16, 16))
    ranges, keys, vals, c = U.gpu_tile_lists(rast)
    assert c.status == 0
    lens = ranges[:, 1] - ranges[:, 0]
    assert lens.max() > 8192, lens.max()
    o = oracle.project(p, view, 16, 16)
    compared, removed = U.compare_tile_lists(keys, vals, gm.n, o, view, (16, 16))
    assert compared > 20_000 and removed <= 0.01 * compared, (compared, removed)
    proj, st, lst, out = oracle.forward_view(p, view, 16, 16)
    mask = U.guard_pixel_mask(view, proj, out, (16, 16))
    img = rast.view_slice(rast.images, 0).cpu().numpy()
    assert np.abs(img - out["image"])[:, ~mask].max() <= IMG_TOL

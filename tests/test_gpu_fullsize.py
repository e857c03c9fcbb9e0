"""Parity at the full sizes of the headline and batched workloads, in the
launch configuration the benchmark times (8x8 tiles, forward batch 128 at one
pixel per thread, backward batch 64 at two pixels per thread, tight tile
rects, the map stored in Z-order).

* 1M Gaussians, SH-3, 1200x680 (the headline): one whole mapping iteration
  against the FP64 oracle's whole iteration on the same seeded inputs (a
  seeded noise target; ~10 s of oracle time): loss, image on every pixel
  outside the guard bands, tile lists bit-exact outside the guarded
  Gaussians, every parameter-gradient group over the Gaussians of
  gpu_util.gradient_keep.
* 500k Gaussians, 16 views of three kinds (the batched form): the batched
  iteration's loss and gradients (summed over the 16 views) against the
  oracle's 16-view iteration (~1 min of oracle time), the images of one
  view of each kind against the oracle's, and the batched iteration against
  the loop of 16 single-view plans.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_13055_gb300 import binding as B
from paper_2409_13055_gb300 import mapping, scenes
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
# Gradients: 1e-4 relative L2 per group, as at the oracle sizes, over the
# Gaussians of gpu_util.gradient_keep.  With a noise target a Gaussian's
# gradient is a random-sign sum over its pixels, so a single pixel where FP32
# and FP64 take its alpha-vs-1/255 decision differently moves it by several
# per cent; the oracle names those Gaussians (guard_g), ~0.2% of the visible
# ones here.  Without that exclusion the groups read 6.9e-5 (means) to
# 3.5e-4 (quaternions), 99% of it from the named Gaussians; with it 1.1e-5 to
# 1.3e-5.  Neither recovering T by division (reading C10) nor the FP32 pixel
# sums contribute at this level: the same errors came out with T carried in
# double precision and with an IEEE reciprocal.
GRAD_TOL = 1e-4
LAUNCH = dict(tile=(8, 8), smem_batch=128, pixels_per_thread=1, smem_batch_bwd=64,
              pixels_per_thread_bwd=2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_13055_gb300 import build
    build.build()
    B.lib()


def test_headline_iteration_matches_oracle():
    p, views, _, lam = scenes.workload("room1M_1200x680")
    p = scenes.z_ordered(p)
    view = views[0]
    target = scenes.random_target(view, scenes.SEED_BASE + 13)
    gm = mapping.GaussianMap(p)
    rast = mapping.fit_instance_capacity(views, gm, headroom=1.5, **LAUNCH)
    m, g = gm.gs_map(), gm.gs_map_grad()
    rast.forward(m)
    rast.loss_l1_ssim(rast.pack([target]), lam)
    rast.render_bwd(m, g)
    torch.cuda.synchronize()
    assert rast.counters().status == 0
    _, keys, vals, _ = U.gpu_tile_lists(rast)
    img = rast.view_slice(rast.images, 0).cpu().numpy()
    loss = rast.loss.item()
    grads = {k: t.cpu().numpy() for k, t in gm.grads().items()}
    del rast, gm
    torch.cuda.empty_cache()

    L, og, renders = oracle.iteration(p, views, [target], lam, 8, 8)
    proj = oracle.project(p, view, 8, 8)
    mask = U.guard_pixel_mask(view, proj, renders[0], (8, 8), params=p)
    assert mask.mean() < 0.02, mask.mean()
    err = np.abs(img - renders[0]["image"])[:, ~mask]
    print(f"1M 1200x680: image max-abs {err.max():.2e} on {100 * (1 - mask.mean()):.2f}% of "
          f"pixels, loss {loss:.8f} vs {L:.8f}")
    assert err.max() <= IMG_TOL
    assert abs(loss - L) <= 1e-5 * abs(L)
    # tile lists: bit-exact outside the Gaussians with a guarded decision
    compared, removed = U.compare_tile_lists(keys, vals, p["means"].shape[0], proj, view, (8, 8))
    print(f"  tile lists: {compared} pairs bit-exact, {removed} pairs of guarded Gaussians removed")
    assert removed <= 0.01 * compared
    keep = U.gradient_keep(p, views, renders, (8, 8))
    vis = proj["tiles_touched"] > 0
    assert (keep & vis).sum() >= 0.95 * vis.sum(), ((keep & vis).sum(), vis.sum())
    errs = U.grad_errors(grads, og, keep)
    for k, e in errs.items():
        print(f"  gradient {k}: rel L2 {e:.2e} over {100 * (keep & vis).sum() / vis.sum():.2f}% "
              f"of the visible Gaussians (all: {U.rel_l2(grads[k], og[k]):.2e})")
    assert all(e <= GRAD_TOL for e in errs.values()), errs


def test_batched16_views_match_oracle_and_per_view_loop():
    p, views, _, lam = scenes.workload("room500k_mixed16")
    p = scenes.z_ordered(p)
    targets = [scenes.random_target(v, scenes.SEED_BASE + 20 + i) for i, v in enumerate(views)]
    out = []
    for batched in (True, False):
        gm = mapping.GaussianMap(p)
        if batched:
            rast = mapping.fit_instance_capacity(views, gm, headroom=1.5, **LAUNCH)
            it = mapping.MappingStep(gm, rast, rast.pack(targets), lam, keep_grads=True)
            it.run()
            torch.cuda.synchronize()
            assert rast.counters().status == 0
            loss = rast.loss.item()
            imgs = {v: rast.view_slice(rast.images, v).cpu().numpy() for v in (0, 6, 12)}
            grads = {k: t.cpu().numpy() for k, t in gm.grads().items()}
        else:
            it = mapping.PerViewLoop(gm, views, targets, lam, keep_grads=True, **LAUNCH)
            it()
            torch.cuda.synchronize()
            loss = sum(r.loss.item() for r in it.rasts)
        out.append((gm.grad.clone().cpu().numpy(), loss))
        del it, gm
        torch.cuda.empty_cache()
    assert abs(out[0][1] - out[1][1]) <= 1e-6 * abs(out[1][1])
    assert U.rel_l2(out[0][0], out[1][0]) < 1e-5
    # the batched iteration against the oracle's 16-view iteration
    L, og, renders = oracle.iteration(p, views, targets, lam, 8, 8)
    assert abs(out[0][1] - L) <= 1e-5 * abs(L), (out[0][1], L)
    keep = U.gradient_keep(p, views, renders, (8, 8))
    errs = U.grad_errors(grads, og, keep)
    print(f"16 views: loss {out[0][1]:.8f} vs {L:.8f}; gradients over {keep.mean() * 100:.2f}% "
          f"of the Gaussians: " + ", ".join(f"{k} {e:.2e}" for k, e in errs.items()))
    assert all(e <= GRAD_TOL for e in errs.values()), errs
    # one view of each kind (640x480 RGB, 752x480 gray, 1200x680 RGB) against the oracle
    for v, img in imgs.items():
        o = renders[v]
        proj = oracle.project(p, views[v], 8, 8)
        mask = U.guard_pixel_mask(views[v], proj, o, (8, 8), params=p)
        assert mask.mean() < 0.02, (v, mask.mean())
        err = np.abs(img - o["image"])[:, ~mask]
        print(f"view {v} {views[v]['width']}x{views[v]['height']}x{views[v]['channels']}: "
              f"max-abs {err.max():.2e}")
        assert err.max() <= IMG_TOL, (v, err.max())


@pytest.mark.parametrize("tile", [(8, 8), (16, 16)])
def test_room200k_iteration_matches_oracle(tile):
    """The 200k-Gaussian room at 640x480 (anisotropic, SH degree 3, L1 + 0.2
    (1 - SSIM), seeded noise target): image, loss, tile lists and every
    gradient group of one iteration against the oracle's, then one Adam step
    against the oracle's Adam on the oracle's gradient."""
    p, views, targets, lam = scenes.workload("room200k_640x480")
    view = views[0]
    launch = dict(LAUNCH, tile=tile) if tile == (8, 8) else dict(tile=tile)
    gm = mapping.GaussianMap(p)
    rast = mapping.fit_instance_capacity(views, gm, headroom=1.5, **launch)
    m, g = gm.gs_map(), gm.gs_map_grad()
    rast.forward(m)
    rast.loss_l1_ssim(rast.pack(targets), lam)
    rast.render_bwd(m, g)
    torch.cuda.synchronize()
    assert rast.counters().status == 0
    _, keys, vals, _ = U.gpu_tile_lists(rast)
    img = rast.view_slice(rast.images, 0).cpu().numpy()
    loss = rast.loss.item()
    grads = {k: t.cpu().numpy() for k, t in gm.grads().items()}
    gm.adam_step()
    torch.cuda.synchronize()
    after = {k: t.cpu().numpy() for k, t in gm.params().items()}

    L, og, renders = oracle.iteration(p, views, targets, lam, *tile)
    proj = oracle.project(p, view, *tile)
    mask = U.guard_pixel_mask(view, proj, renders[0], tile, params=p)
    assert mask.mean() < 0.02, mask.mean()
    err = np.abs(img - renders[0]["image"])[:, ~mask]
    assert err.max() <= IMG_TOL, err.max()
    assert abs(loss - L) <= 1e-5 * abs(L), (loss, L)
    compared, removed = U.compare_tile_lists(keys, vals, p["means"].shape[0], proj, view, tile)
    assert compared > 100_000 and removed <= 0.01 * compared, (compared, removed)
    keep = U.gradient_keep(p, views, renders, tile)
    vis = proj["tiles_touched"] > 0
    assert (keep & vis).sum() >= 0.95 * vis.sum()
    errs = U.grad_errors(grads, og, keep)
    print(f"200k 640x480 {tile}: image max-abs {err.max():.2e}, loss {loss:.8f} vs {L:.8f}, "
          f"{compared} list pairs bit-exact, gradients " +
          ", ".join(f"{k} {e:.2e}" for k, e in errs.items()))
    assert all(e <= GRAD_TOL for e in errs.values()), errs
    # one Adam step (3DGS default rates) from zero moments on the GPU's own
    # gradient, against the oracle's Adam on the same gradient; with eps =
    # 1e-15 a first step moves a parameter by ~lr sign(g) for any |g| >> eps,
    # so elements whose g^2 leaves the FP32 normal range (|g| < 1e-19) are
    # left out
    lr = dict(zip(oracle.PARAM_GROUPS, (1.6e-4, 5e-3, 1e-3, 0.05, None)))
    for k in oracle.PARAM_GROUPS:
        p0 = np.asarray(p[k], np.float64).copy()
        gk = grads[k].astype(np.float64)
        mm, vv = np.zeros_like(p0), np.zeros_like(p0)
        if k == "sh":
            for c, rate in ((slice(0, 1), 2.5e-3), (slice(1, None), 2.5e-3 / 20)):
                pc = np.ascontiguousarray(p0[c])
                oracle.adam(pc, gk[c], np.zeros_like(pc), np.zeros_like(pc), rate, 1)
                p0[c] = pc
        else:
            oracle.adam(p0, gk, mm, vv, lr[k], 1)
        ok = (np.abs(gk) >= 1e-19) | (gk == 0)
        assert ok.mean() > 0.99, (k, ok.mean())
        # FP32 p - lr x: rounding of the FP32 operands (|p| and the step lr)
        before = np.asarray(p[k], np.float64)
        rate = np.full_like(before, lr[k]) if k != "sh" else np.concatenate(
            [np.full_like(before[:1], 2.5e-3), np.full_like(before[1:], 2.5e-3 / 20)])
        tol = 1.2e-7 * (np.abs(before) + rate) + 1e-6 * rate
        err = np.abs(after[k].astype(np.float64) - p0)
        assert np.all(err[ok] <= tol[ok]), (k, float((err - tol)[ok].max()))

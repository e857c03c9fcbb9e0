"""GPU parity of the adaptive density control (paper Sec. III-B: AbsGS
homodirectional statistic, clone / split / prune) against the FP64 oracle.

Bars: the homodirectional sums per (view, Gaussian) within 1e-4 relative L2
(the gradient bar); the accumulated statistic within 1e-6 relative of the
oracle's accumulation of the GPU's own per-view sums; categories exact on
inputs that keep every decision 1% away from its threshold; the new map's
copied values bit-exact and the split children's means within 1e-6
relative (FP32 rotation of a standard-normal offset).
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_13055_gb300 import build
    build.build()
    B.lib()


@pytest.mark.parametrize("tile,ppt", [((16, 16), 1), ((8, 8), 2)])
def test_homodirectional_sums_and_statistic(tile, ppt):
    p = scenes.room_scene(20_000, seed=31)
    views = [scenes.camera(160, 120, 131.25, 131.25),
             dict(scenes.camera(188, 120, 115.0, 115.0, channels=1))]
    targets = [scenes.random_target(v, 70 + i) for i, v in enumerate(views)]
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer(views, gm.n, instance_capacity=1 << 21, tile=tile,
                              pixels_per_thread=ppt, pixels_per_thread_bwd=ppt, density_stats=True)
    plain = mapping.Rasterizer(views, gm.n, instance_capacity=1 << 21, tile=tile,
                               pixels_per_thread=ppt, pixels_per_thread_bwd=ppt)
    out = []
    for r in (rast, plain):
        g = torch.zeros_like(gm.grad)
        m = gm.gs_map()
        r.forward(m)
        r.loss_l1_ssim(r.pack(targets), 0.2)
        r.render_bwd(m, gm._struct(g))
        torch.cuda.synchronize()
        out.append(g.cpu().numpy())
    # the extra sums change only the order of the reduction of the others
    assert U.rel_l2(out[0], out[1]) < 1e-6
    n = gm.n
    absg = rast.buffer(B.GS_BUF_ABSGRAD, torch.float32)[: 2 * 2 * n].view(2, n, 2).cpu().numpy()
    touched = rast.buffer(B.GS_BUF_TOUCHED, torch.int32)[: 2 * n].view(2, n).cpu().numpy()
    accum = torch.zeros(n, device="cuda")
    denom = torch.zeros(n, device="cuda")
    rast.densify_stats(n, accum, denom)
    torch.cuda.synchronize()
    oa, od = np.zeros(n), np.zeros(n)
    for v, view in enumerate(views):
        proj, st, lst, o = oracle.forward_view(p, view, tile[0], tile[1])
        _, dimg = oracle.loss_l1_ssim(o["image"], targets[v], 0.2)
        g2d = oracle.render_bwd(proj, st, lst, view, dimg / 2, tile[0], tile[1])
        assert U.rel_l2(absg[v], g2d["dmean2d_abs"]) < 1e-4
        np.testing.assert_array_equal(touched[v] > 0, proj["tiles_touched"] > 0)
        oracle.densify_stats(oa, od, view, touched[v], absg[v].astype(np.float64))
    np.testing.assert_array_equal(denom.cpu().numpy(), od)
    np.testing.assert_allclose(accum.cpu().numpy(), oa, rtol=1e-6, atol=1e-30)


def _map_with_margins(n, seed):
    """A map and statistic whose every decision is >= 1% from its threshold:
    opacity vs 0.005, mean statistic vs 4e-4, largest scale vs 0.01 extent."""
    rng = np.random.default_rng(seed)
    p = scenes.tiny_scene(n, 64, 48, seed=seed, sh_degree=3)[0]
    op = np.where(rng.uniform(size=n) < 0.1, rng.uniform(0.001, 0.0049, n),
                  rng.uniform(0.01, 0.9, n))
    p["opacity_logits"] = np.log(op / (1 - op)).astype(np.float32)
    smax = np.where(rng.uniform(size=n) < 0.5, rng.uniform(0.002, 0.0099, n),
                    rng.uniform(0.0101, 0.05, n))
    ls = np.log(smax)[:, None] - rng.uniform(0.0, 1.0, (n, 3))
    ls[np.arange(n), rng.integers(0, 3, n)] = np.log(smax)
    p["log_scales"] = ls.astype(np.float32)
    denom = rng.integers(0, 4, n).astype(np.float32)
    stat = np.where(rng.uniform(size=n) < 0.4, rng.uniform(4.05e-4, 2e-3, n),
                    rng.uniform(0.0, 3.95e-4, n))
    accum = (stat * denom).astype(np.float32)
    return p, accum, denom


def test_densify_matches_oracle():
    n = 3001  # several blocks and a ragged tail
    p, accum, denom = _map_with_margins(n, 5)
    gm = mapping.GaussianMap(p)
    rng = np.random.default_rng(9)
    gm.m.uniform_(-1.0, 1.0)
    gm.v.uniform_(0.0, 1.0)
    samples = rng.normal(size=(n, 2, 3)).astype(np.float32)
    before = gm.to_numpy()
    mom = {}
    for k in oracle.PARAM_GROUPS:
        mom[k] = (gm._views(gm.m)[k].cpu().numpy().astype(np.float64),
                  gm._views(gm.v)[k].cpu().numpy().astype(np.float64))
    cat = oracle.densify_categories(before, accum, denom, extent=1.0)
    kept, cloned, split = gm.densify(torch.tensor(accum, device="cuda"),
                                     torch.tensor(denom, device="cuda"),
                                     torch.tensor(samples, device="cuda"), extent=1.0)
    assert (kept, cloned, split) == (int(np.sum((cat == 1) | (cat == 2))), int(np.sum(cat == 2)),
                                     int(np.sum(cat == 3)))
    assert min(np.sum(cat == c) for c in range(4)) > 20  # every category exercised
    want, want_m = oracle.densify_apply(before, mom, cat, samples.astype(np.float64))
    got = gm.to_numpy()
    assert gm.n == kept + cloned + 2 * split == want["means"].shape[0]
    base = kept + cloned
    for k in ("quats", "opacity_logits", "sh"):
        np.testing.assert_array_equal(got[k], want[k].astype(np.float32), err_msg=k)
    for k in ("means", "log_scales"):
        np.testing.assert_array_equal(got[k][:base], want[k][:base].astype(np.float32))
    # children's log-scales: one FP32 subtraction of log(1.6)
    np.testing.assert_allclose(got["log_scales"][base:], want["log_scales"][base:], rtol=0,
                               atol=1e-6)
    err = np.abs(got["means"][base:] - want["means"][base:])
    assert np.max(err / (np.abs(want["means"][base:]) + 1e-3)) < 1e-6
    for k in oracle.PARAM_GROUPS:
        gmk = gm._views(gm.m)[k].cpu().numpy()
        gvk = gm._views(gm.v)[k].cpu().numpy()
        np.testing.assert_array_equal(gmk, want_m[k][0].astype(np.float32), err_msg=k)
        np.testing.assert_array_equal(gvk, want_m[k][1].astype(np.float32), err_msg=k)


def test_densify_inside_a_mapping_loop():
    """Iterations with the statistic accumulated inside the captured step,
    then density control, then more iterations on the new map: sizes agree
    with the categories of the accumulated statistic, the loss stays finite
    and the device status clean."""
    p = scenes.room_scene(30_000, seed=41)
    view = scenes.camera(200, 150, 160.0, 160.0)
    target = scenes.random_target(view, 77)
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer([view], gm.n, instance_capacity=1 << 21, density_stats=True)
    accum = torch.zeros(gm.n, device="cuda")
    denom = torch.zeros(gm.n, device="cuda")
    step = mapping.MappingStep(gm, rast, rast.pack([target]), 0.2, stats=(accum, denom))
    step.capture(warmup=1)
    for _ in range(4):
        step()
    torch.cuda.synchronize()
    cat = oracle.densify_categories(gm.to_numpy(), accum.cpu().numpy(), denom.cpu().numpy(), 1.0)
    samples = torch.randn(gm.n, 2, 3, device="cuda")
    kept, cloned, split = gm.densify(accum, denom, samples, extent=1.0)
    assert kept == int(np.sum((cat == 1) | (cat == 2))) and split == int(np.sum(cat == 3))
    assert cloned + split > 0
    rast2 = mapping.fit_instance_capacity([view], gm, density_stats=True)
    step2 = mapping.MappingStep(gm, rast2, rast2.pack([target]), 0.2)
    for _ in range(3):
        step2()
    torch.cuda.synchronize()
    assert math.isfinite(rast2.loss.item())
    assert rast2.counters().status == 0

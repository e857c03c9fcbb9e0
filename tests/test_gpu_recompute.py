"""The recompute (checkpointing) mode: a plan whose workspace holds one view's
projection and binning, views run through it one pass at a time, and the
backward repeats each view's projection and binning before its adjoint
(no counterpart in the paper; the mode the mapping of large maps and long
keyframe windows uses).

Checks: the same images, loss and gradients as the plan that keeps every
view's projection -- bit for bit in a deterministic one-view plan -- with a
smaller workspace; the autograd Function with several renders pending at once on
rasterisers that share one workspace; the error of a backward whose forward
was overwritten in a plan that keeps the projection.
"""
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


def posed(view, seed, trans=0.2, ang=10.0):
    R, t = scenes.random_pose(np.random.default_rng(seed), trans, ang)
    return dict(view, R=R, t=t * 0.3)


def _case():
    p = scenes.room_scene(30_000, seed=51)
    views = [scenes.camera(160, 120, 131.25, 131.25),
             posed(scenes.camera(188, 120, 115.0, 115.0, channels=1), 8),
             posed(scenes.camera(200, 112, 100.0, 100.0), 9)]
    targets = [scenes.random_target(v, 60 + i) for i, v in enumerate(views)]
    return p, views, targets


def _iteration(p, views, targets, **kw):
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer(views, gm.n, instance_capacity=1 << 20, tile=(8, 8),
                              pixels_per_thread_bwd=2, bg=(0.1, 0.2, 0.3), **kw)
    m, g = gm.gs_map(), gm.gs_map_grad()
    rast.forward(m)
    rast.loss_l1_ssim(rast.pack(targets), 0.2)
    rast.render_bwd(m, g)
    torch.cuda.synchronize()
    c = rast.counters()
    assert c.status == 0, c.status
    return dict(img=rast.images.clone(), T=rast.final_T.clone(), last=rast.last_idx.clone(),
                loss=rast.loss.item(), grad=gm.grad.clone(), ws=rast.workspace_bytes, gm=gm)


@pytest.mark.parametrize("nviews,per_pass", [(1, 1), (3, 1), (3, 2)])
def test_recompute_plan_equals_kept_projection(nviews, per_pass):
    p, views, targets = _case()
    views, targets = views[:nviews], targets[:nviews]
    for det in (True, False):
        keep = _iteration(p, views, targets, deterministic=det)
        rec = _iteration(p, views, targets, deterministic=det, recompute=per_pass)
        assert torch.equal(rec["img"], keep["img"]) and torch.equal(rec["T"], keep["T"])
        assert torch.equal(rec["last"], keep["last"])
        assert rec["loss"] == keep["loss"]
        if det and nviews == 1:
            # the deterministic adjoint adds the same numbers in the same order
            assert torch.equal(rec["grad"], keep["grad"])
        elif det:
            # several views: the plan that keeps them all sums a Gaussian's
            # views in registers (with fused multiply-adds for the SH terms),
            # the passes through the gradient buffer, so the last bits differ
            assert U.rel_l2(rec["grad"].cpu().numpy(), keep["grad"].cpu().numpy()) < 1e-6
        else:
            assert U.rel_l2(rec["grad"].cpu().numpy(), keep["grad"].cpu().numpy()) < 1e-6
        if nviews > per_pass:
            # the projection and binning buffers of per_pass views instead of
            # three (~200 B per (view, Gaussian)); the instance buffers, of
            # the same capacity here, are the same size
            assert keep["ws"] - rec["ws"] >= (nviews - per_pass) * p["means"].shape[0] * 150, (
                rec["ws"], keep["ws"])
    # and the recompute plan against the oracle
    L, og, renders = oracle.iteration(p, views, targets, 0.2, 8, 8, bg=(0.1, 0.2, 0.3))
    assert abs(rec["loss"] - L) <= 1e-5 * abs(L)
    keep_g = U.gradient_keep(p, views, renders, (8, 8))
    errs = U.grad_errors({k: t.cpu().numpy() for k, t in rec["gm"].grads().items()}, og, keep_g)
    assert all(e <= 1e-4 for e in errs.values()), errs


def test_mapping_step_with_recompute_rasteriser():
    """MappingStep over a recompute rasteriser of three views (passes in one
    CUDA graph) gives the batched step's loss, gradients and update."""
    p, views, targets = _case()
    out = []
    for rec in (False, True):
        gm = mapping.GaussianMap(p)
        rast = mapping.fit_instance_capacity(views, gm, tile=(8, 8), pixels_per_thread_bwd=2,
                                             recompute=2 if rec else 0)
        step = mapping.MappingStep(gm, rast, rast.pack(targets), 0.2, keep_grads=True)
        assert step.recompute == rec
        step.capture(warmup=1)
        start = gm.data.clone()
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        assert rast.counters().status == 0
        out.append((rast.loss.item(), gm.grad.clone().cpu().numpy(),
                    (gm.data - start).cpu().numpy(), rast.workspace_bytes))
    assert abs(out[0][0] - out[1][0]) <= 1e-6 * abs(out[0][0])
    assert U.rel_l2(out[1][1], out[0][1]) < 1e-5
    assert U.rel_l2(out[1][2], out[0][2]) < 1e-3
    assert out[1][3] < out[0][3]


def test_autograd_renders_pending_on_a_shared_workspace():
    """Three GSRender calls, each on its own one-view recompute rasteriser,
    all sharing one workspace, summed into one loss before a single
    backward: the gradient equals the sum of the three single-render
    gradients."""
    p, views, targets = _case()
    gm = mapping.GaussianMap(p)
    rasts = [mapping.Rasterizer([v], gm.n, instance_capacity=1 << 20, recompute=True)
             for v in views]
    shared = torch.zeros(max(r.workspace_bytes for r in rasts), dtype=torch.uint8,
                         device="cuda")
    rasts = [mapping.Rasterizer([v], gm.n, instance_capacity=1 << 20, recompute=True,
                                workspace=shared) for v in views]
    P = gm.params()
    names = ("means", "log_scales", "quats", "opacity_logits", "sh")

    def leaves():
        return [P[k].detach().clone().contiguous().requires_grad_(True) for k in names]

    tg = [torch.as_tensor(t).cuda().reshape(-1) for t in targets]
    x = leaves()
    loss = sum(mapping.L1SSIMLoss.apply(mapping.GSRender.apply(*x, r), t, r, 0.2)
               for r, t in zip(rasts, tg))
    loss.backward()
    total = [l.grad.clone() for l in x]
    want = [torch.zeros_like(t) for t in total]
    L = 0.0
    for r, t in zip(rasts, tg):
        y = leaves()
        li = mapping.L1SSIMLoss.apply(mapping.GSRender.apply(*y, r), t, r, 0.2)
        li.backward()
        L += li.item()
        for w, l in zip(want, y):
            w += l.grad
    assert abs(loss.item() - L) <= 1e-6 * abs(L)
    for a, b in zip(total, want):
        assert U.rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    # against the oracle, view by view summed, over the Gaussians clear of
    # guarded decisions in every view
    og = oracle.zero_grads(p)
    keep = np.ones(gm.n, bool)
    for v, t in zip(views, targets):
        _, g1, r1 = oracle.iteration(p, [v], [t], 0.2)
        keep &= U.gradient_keep(p, [v], r1)
        for k in og:
            og[k] += g1[k]
    assert keep.mean() > 0.95
    errs = U.grad_errors(dict(zip(names, (g.cpu().numpy() for g in total))), og, keep)
    assert all(e <= 1e-4 for e in errs.values()), errs


def test_kept_projection_backward_after_another_forward_raises():
    p, views, targets = _case()
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer(views[:1], gm.n, instance_capacity=1 << 20)
    P = gm.params()
    x = [P[k].detach().clone().contiguous().requires_grad_(True)
         for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    img1 = mapping.GSRender.apply(*x, rast)
    img2 = mapping.GSRender.apply(*x, rast)
    img2.sum().backward(retain_graph=True)  # the latest forward: fine
    with pytest.raises(RuntimeError, match="another forward"):
        img1.sum().backward()

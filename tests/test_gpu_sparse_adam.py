"""GPU parity of the visibility-masked ("sparse") Adam variant against the
oracle's masked Adam (the dense Adam of paper Sec. IV-A on the visible
Gaussians' elements, the rest untouched).

Bars: 1e-6 relative per element on visible elements (the dense Adam bar);
invisible elements and the group padding bit-identical to their inputs; the
visibility bytes exact against the oracle's projection.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_13055_gb300 import binding as B
from paper_2409_13055_gb300 import mapping, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_13055_gb300 import build
    build.build()
    B.lib()


def test_visibility_matches_projection():
    p = scenes.room_scene(20_000, seed=31)
    views = [scenes.camera(160, 120, 131.25, 131.25),
             dict(scenes.camera(188, 120, 115.0, 115.0, channels=1))]
    gm = mapping.GaussianMap(p)
    rast = mapping.Rasterizer(views, gm.n, instance_capacity=1 << 21)
    rast.project(gm.gs_map())
    vis = torch.zeros(gm.n, dtype=torch.uint8, device="cuda")
    rast.visibility(gm.n, vis)
    want = np.zeros(gm.n, bool)
    for v in views:
        want |= oracle.project(p, v)["tiles_touched"] > 0
    assert 0.05 < want.mean() < 0.95
    np.testing.assert_array_equal(vis.cpu().numpy().astype(bool), want)


def test_sparse_adam_matches_masked_oracle():
    n = 1001
    p = scenes.tiny_scene(n, 64, 48, seed=3, sh_degree=3)[0]
    gm = mapping.GaussianMap(p)
    rng = np.random.default_rng(4)
    # gradient statistics of a running optimisation: |m| ~ |g| ~ 1e-3, v ~ g^2
    gm.grad.copy_(torch.tensor(rng.normal(0, 1e-3, size=gm.total).astype(np.float32)))
    gm.m.copy_(torch.tensor(rng.normal(0, 1e-3, size=gm.total).astype(np.float32)))
    gm.v.copy_(torch.tensor(rng.uniform(1e-7, 2e-6, size=gm.total).astype(np.float32)))
    vis = rng.uniform(size=n) < 0.45
    # element -> Gaussian index through the map's own group views
    owner = torch.full((gm.total,), -1.0, device="cuda")
    for k, t in gm._views(owner).items():
        idx = torch.arange(n, dtype=torch.float32, device="cuda")
        if k == "sh":
            t.copy_(idx.view(1, n, 1).expand_as(t))
        elif t.dim() == 2:
            t.copy_(idx.view(n, 1).expand_as(t))
        else:
            t.copy_(idx)
    owner = owner.cpu().numpy().astype(np.int64)
    offs, rates = gm.adam_groups()
    P, G, M, V = (x.cpu().numpy().astype(np.float64) for x in (gm.data, gm.grad, gm.m, gm.v))
    P0 = P.copy()
    vis_t = torch.tensor(vis.astype(np.uint8), device="cuda")
    for step in (1, 2):
        gm.adam_step(visible=vis_t)
        for k in range(len(rates)):
            sl = slice(offs[k], offs[k + 1])
            mask = (owner[sl] >= 0) & vis[np.maximum(owner[sl], 0)]
            # the betas as the kernel receives them (FP32 0.9 and 0.999)
            oracle.adam_masked(P[sl], G[sl], M[sl], V[sl], rates[k], step, mask,
                               b1=float(np.float32(0.9)), b2=float(np.float32(0.999)))
    torch.cuda.synchronize()
    got = gm.data.cpu().numpy()
    touched = (owner >= 0) & vis[np.maximum(owner, 0)]
    np.testing.assert_array_equal(got[~touched], P0[~touched].astype(np.float32))
    np.testing.assert_allclose(got[touched], P[touched], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(gm.m.cpu().numpy()[touched], M[touched], rtol=1e-6, atol=1e-7)
    assert int(gm.step.item()) == 2

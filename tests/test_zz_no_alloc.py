"""gs_loss_l1_ssim_noalloc: the loss for callers that cannot allocate device
memory (no workspace), using the library's fixed scratch array.

Collected last on purpose: it exercises state that lives for the whole
process (the array and its contents, on every device that loaded the
library's device code), and a failure here should not hide any other test's
result.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2409_13055_gb300 import binding as B
from paper_2409_13055_gb300 import mapping, scenes


@pytest.fixture(scope="module")
def lib():
    from paper_2409_13055_gb300 import build
    build.build()
    return B.lib()


def _plan(views):
    cfg = B.gs_config(16, 16, 128, 0, 0, 0, 0.2, (B.c_float * 3)(0, 0, 0))
    return B.gs_plan_init(cfg, [mapping.make_view(v) for v in views], 16, 1024)


def test_rejects_plans_beyond_the_fixed_scratch(lib):
    """2^20 values at most: a 1200x680 RGB view (2.45M values) is refused
    before anything touches the GPU."""
    plan = _plan([scenes.camera(1200, 680, 600.0, 600.0)])
    p = ctypes.c_void_p(256)
    st = lib.gs_loss_l1_ssim_noalloc(ctypes.byref(plan), p, p, 0.2, 1.0, p, p, None)
    assert st == B.GS_ERR_CAPACITY


@pytest.mark.gpu
def test_matches_workspace_entry_point_on_two_calls(lib):
    """Two calls in a row (different images, different plans) through the
    C-ABI equal gs_loss_l1_ssim with a workspace, within the loss tests'
    tolerance; the second call must not see the first call's scratch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = [
        ([scenes.camera(640, 480, 525.0, 525.0)], 0.2, 1.0),
        ([scenes.camera(300, 170, 150.0, 150.0), scenes.camera(188, 120, 115.0, 115.0, channels=1)],
         0.8, 0.5),
    ]
    rng = np.random.default_rng(7)
    for views, lam, weight in cases:
        rast = mapping.Rasterizer(views, 16, instance_capacity=1024)
        img = torch.from_numpy(rng.uniform(0, 1, rast.total_values).astype(np.float32)).cuda()
        tgt = torch.from_numpy(rng.uniform(0, 1, rast.total_values).astype(np.float32)).cuda()
        rast.loss_l1_ssim(tgt, lam, view_weight=weight, images=img)
        ref_loss, ref_dL = rast.loss.clone(), rast.dL.clone()
        loss = torch.full((1,), -1.0, device="cuda")
        dL = torch.full_like(ref_dL, float("nan"))
        st = B.gs_loss_l1_ssim_noalloc(rast.plan, img, tgt, lam, weight, loss, dL)
        assert st == B.GS_OK, B.gs_status_string(st)
        torch.cuda.synchronize()
        assert abs(loss.item() - ref_loss.item()) <= 1e-5 * max(1.0, abs(ref_loss.item()))
        assert torch.isfinite(dL).all()
        err = (dL - ref_dL).abs().max().item()
        assert err <= 1e-5 * ref_dL.abs().max().item()

"""Host-side checks of the C-ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/gs.h declares, and its
host-only entry points validate their arguments and size workspaces."""
import ctypes
import shutil

import pytest

from paper_2409_13055_gb300 import binding as B
from paper_2409_13055_gb300 import build as gsbuild
from paper_2409_13055_gb300 import mapping, scenes

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not __import__("os").path.exists(
    "/usr/local/cuda/bin/nvcc"), reason="nvcc is needed to build the library")


@pytest.fixture(scope="module")
def lib():
    gsbuild.build()
    return B.lib()


def test_exports_every_declared_function(lib):
    names = B.header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B._SIGNATURES), set(names) ^ set(B._SIGNATURES)


def test_struct_sizes_match_header():
    assert ctypes.sizeof(B.gs_view) == 80
    assert ctypes.sizeof(B.gs_config) == 56
    assert ctypes.sizeof(B.gs_densify_config) == 32
    assert ctypes.sizeof(B.gs_counters) == 32
    assert ctypes.sizeof(B.gs_plan) == 8 * B.GS_PLAN_WORDS


def _cfg(tw=16, th=16, batch=128, near=0.2, ppt=0, batch_bwd=0, ppt_bwd=0, recompute=0):
    return B.gs_config(tw, th, batch, ppt, batch_bwd, ppt_bwd, near, (B.c_float * 3)(0, 0, 0),
                       0, 0, 1, recompute)


def _views(*sizes):
    return [mapping.make_view(scenes.camera(w, h, 500.0, 500.0, channels=c)) for (w, h, c) in sizes]


def test_plan_layout_and_offsets(lib):
    vs = _views((640, 480, 3), (752, 480, 1), (1200, 680, 3))
    plan = B.gs_plan_init(_cfg(), vs, 1000, 100000)
    tot = B.gs_plan_totals(plan)
    assert tot["total_values"] == 640 * 480 * 3 + 752 * 480 + 1200 * 680 * 3
    assert tot["total_pixels"] == 640 * 480 + 752 * 480 + 1200 * 680
    assert tot["total_tiles"] == 40 * 30 + 47 * 30 + 75 * 43
    v2 = B.gs_plan_view(plan, 2)
    assert v2["value_offset"] == 640 * 480 * 3 + 752 * 480
    assert v2["pixel_offset"] == 640 * 480 + 752 * 480
    assert v2["tile_offset"] == 40 * 30 + 47 * 30
    assert (v2["tiles_x"], v2["tiles_y"]) == (75, 43)
    ws = B.gs_plan_workspace_bytes(plan)
    seen = []
    for b in range(10):
        off, nbytes = B.gs_plan_buffer(plan, b)
        assert off % 256 == 0 and off + nbytes <= ws
        seen.append((off, nbytes))


@pytest.mark.parametrize("cfg,views,ncap,icap,err", [
    (dict(tw=12), [(64, 64, 3)], 10, 100, B.GS_ERR_UNSUPPORTED),
    (dict(tw=64, th=8), [(64, 64, 3)], 10, 100, B.GS_ERR_UNSUPPORTED),
    (dict(batch=48), [(64, 64, 3)], 10, 100, B.GS_ERR_UNSUPPORTED),
    (dict(near=0.0), [(64, 64, 3)], 10, 100, B.GS_ERR_INVALID),
    (dict(ppt=3), [(64, 64, 3)], 10, 100, B.GS_ERR_UNSUPPORTED),
    (dict(tw=8, th=8, ppt=4), [(64, 64, 3)], 10, 100, B.GS_ERR_UNSUPPORTED),
    (dict(ppt_bwd=3), [(64, 64, 3)], 10, 100, B.GS_ERR_UNSUPPORTED),
    (dict(batch_bwd=40), [(64, 64, 3)], 10, 100, B.GS_ERR_UNSUPPORTED),
    (dict(), [(64, 64, 2)], 10, 100, B.GS_ERR_INVALID),
    (dict(), [(0, 64, 3)], 10, 100, B.GS_ERR_INVALID),
    (dict(), [(64, 64, 3)], 0, 100, B.GS_ERR_INVALID),
    (dict(), [(64, 64, 3)], 10, 0, B.GS_ERR_INVALID),
])
def test_plan_init_rejects(lib, cfg, views, ncap, icap, err):
    plan = B.gs_plan()
    arr = (B.gs_view * len(views))(*_views(*views))
    st = lib.gs_plan_init(ctypes.byref(plan), ctypes.byref(_cfg(**cfg)), len(views), arr, ncap,
                          icap)
    assert st == err


def test_calls_reject_bad_arguments_without_launching(lib):
    plan = B.gs_plan_init(_cfg(), _views((64, 48, 3)), 10, 1000)
    nullmap = B.gs_map(None, None, None, None, None, 10, 0)
    assert lib.gs_project(ctypes.byref(plan), ctypes.byref(nullmap), None, None, None) == \
        B.GS_ERR_INVALID
    assert lib.gs_bin_sort(ctypes.byref(plan), 0, ctypes.c_void_p(256), None) == B.GS_ERR_INVALID
    bad = B.gs_plan()  # never initialised
    assert lib.gs_render_fwd(ctypes.byref(bad), ctypes.c_void_p(256), ctypes.c_void_p(256),
                             ctypes.c_void_p(256), ctypes.c_void_p(256), None) == B.GS_ERR_INVALID
    assert lib.gs_loss_l1_ssim(ctypes.byref(plan), ctypes.c_void_p(256), ctypes.c_void_p(256),
                               1.5, 1.0, ctypes.c_void_p(256), ctypes.c_void_p(256),
                               ctypes.c_void_p(256), None) == B.GS_ERR_INVALID
    offs = (B.c_int64 * 2)(0, 5)
    lrs = (B.c_float * 1)(0.1)
    p = ctypes.c_void_p(256)
    assert lib.gs_adam_step(p, p, p, p, 6, 1, offs, lrs, 0.9, 0.999, 1e-15, p, None) == \
        B.GS_ERR_INVALID  # offsets do not end at n
    assert lib.gs_adam_step(p, p, p, p, 5, 1, offs, lrs, 1.0, 0.999, 1e-15, p, None) == \
        B.GS_ERR_INVALID  # beta1 = 1
    assert B.gs_status_string(B.GS_ERR_CAPACITY).startswith("GS_ERR_CAPACITY")


def test_recompute_plans_hold_one_view_and_run_passes(lib):
    """A recompute plan lays the projection and binning out for one view
    (the loss maps sharing those bytes), so its workspace is smaller; its
    view passes share the layout and address each view's images; the whole
    plan of several views is refused by the per-view calls, which take
    passes."""
    vs = _views((640, 480, 3), (752, 480, 1), (1200, 680, 3))
    n, icap = 200_000, 2_000_000
    full = B.gs_plan_init(_cfg(tw=8, th=8), vs, n, icap)
    rec = B.gs_plan_init(_cfg(tw=8, th=8, recompute=1), vs, n, icap)
    wf, wr = B.gs_plan_workspace_bytes(full), B.gs_plan_workspace_bytes(rec)
    # (V - 1) views x ~200 B per Gaussian saved at least (the instance
    # capacity, the same here, is one view's in the recompute plan)
    assert wr < wf - 2 * n * 180, (wf, wr)
    one = B.gs_plan_init(_cfg(tw=8, th=8), vs[2:], n, icap)
    assert wr <= B.gs_plan_workspace_bytes(one) + 256
    for v in range(3):
        ps = B.gs_plan_view_pass(rec, v)
        assert B.gs_plan_workspace_bytes(ps) == wr
        assert B.gs_plan_view(ps, 0)["value_offset"] == B.gs_plan_view(rec, v)["value_offset"]
        assert B.gs_plan_totals(ps)["total_tiles"] == \
            B.gs_plan_view(rec, v)["tiles_x"] * B.gs_plan_view(rec, v)["tiles_y"]
        for b in range(B.GS_BUF_ABSGRAD + 1):
            assert B.gs_plan_buffer(ps, b) == B.gs_plan_buffer(rec, b) or b in (
                B.GS_BUF_TILE_KEYS, B.GS_BUF_TILE_VALUES)
    assert B.gs_plan_passes(rec) == 3 and B.gs_plan_passes(full) == 1
    # passes of two views: [0, 1] and [2]
    two = B.gs_plan_init(_cfg(tw=8, th=8, recompute=2), vs, n, icap)
    assert B.gs_plan_passes(two) == 2
    p0, p1 = B.gs_plan_view_pass(two, 0), B.gs_plan_view_pass(two, 1)
    v1 = B.gs_plan_view(rec, 1)
    assert B.gs_plan_totals(p0)["total_tiles"] == 80 * 60 + 94 * 60  # 640x480 and 752x480 at 8x8
    assert B.gs_plan_view(p0, 1)["tile_offset"] == 80 * 60
    assert B.gs_plan_view(p0, 1)["value_offset"] == v1["value_offset"]
    assert B.gs_plan_view(p1, 0)["value_offset"] == B.gs_plan_view(rec, 2)["value_offset"]
    assert wr < B.gs_plan_workspace_bytes(two) < wf
    bad = B.gs_plan()
    assert lib.gs_plan_view_pass(ctypes.byref(two), 2, ctypes.byref(bad)) == B.GS_ERR_INVALID
    assert lib.gs_plan_view_pass(ctypes.byref(full), 0, ctypes.byref(bad)) == B.GS_ERR_INVALID
    assert lib.gs_plan_view_pass(ctypes.byref(rec), 3, ctypes.byref(bad)) == B.GS_ERR_INVALID
    ps = B.gs_plan_view_pass(rec, 1)
    assert lib.gs_plan_view_pass(ctypes.byref(ps), 0, ctypes.byref(bad)) == B.GS_ERR_INVALID
    p = ctypes.c_void_p(256)
    m = B.gs_map(p, p, p, p, p, 10, 3)
    g = B.gs_map_grad(p, p, p, p, p)
    for plan in (rec,):  # every per-view call refuses the whole plan (nothing launched)
        assert lib.gs_project(ctypes.byref(plan), ctypes.byref(m), p, p, None) == B.GS_ERR_INVALID
        assert lib.gs_bin_sort(ctypes.byref(plan), 10, p, None) == B.GS_ERR_INVALID
        assert lib.gs_render_fwd(ctypes.byref(plan), p, p, p, p, None) == B.GS_ERR_INVALID
        assert lib.gs_render_bwd_pixels(ctypes.byref(plan), p, p, p, p, None) == \
            B.GS_ERR_INVALID
        assert lib.gs_project_bwd(ctypes.byref(plan), ctypes.byref(m), p, p, ctypes.byref(g), 0,
                                  None) == B.GS_ERR_INVALID
    # ... and the calls that need every view at once refuse a pass
    assert lib.gs_project_bwd_groups(ctypes.byref(ps), ctypes.byref(m), p, p, ctypes.byref(g), p,
                                     None) == B.GS_ERR_INVALID
    assert lib.gs_visibility(ctypes.byref(ps), 10, p, p, None) == B.GS_ERR_INVALID


def test_deterministic_plans_need_one_warp_per_tile(lib):
    views = _views((64, 48, 3))
    ok = B.gs_config(8, 8, 64, 1, 32, 2, 0.2, (B.c_float * 3)(0, 0, 0), 0, 1)
    bad = B.gs_config(16, 16, 64, 1, 64, 1, 0.2, (B.c_float * 3)(0, 0, 0), 0, 1)
    plan = B.gs_plan()
    arr = (B.gs_view * 1)(*views)
    assert lib.gs_plan_init(ctypes.byref(plan), ctypes.byref(ok), 1, arr, 10, 1000) == B.GS_OK
    assert lib.gs_plan_init(ctypes.byref(plan), ctypes.byref(bad), 1, arr, 10, 1000) == \
        B.GS_ERR_UNSUPPORTED


def test_density_control_rejects_bad_arguments_without_launching(lib):
    p = ctypes.c_void_p(256)
    plan = B.gs_plan_init(_cfg(), _views((64, 48, 3)), 10, 1000)  # no density_stats
    assert lib.gs_densify_stats(ctypes.byref(plan), 10, p, p, p, None) == B.GS_ERR_INVALID
    assert lib.gs_densify_scratch_bytes(0) == 0
    assert lib.gs_densify_scratch_bytes(257) == 6 * 2 * 4 + 256
    good = B.gs_densify_config(0.0004, 0.01, 0.005, 1.6, 1.0)
    badcfg = B.gs_densify_config(0.0004, 0.01, 0.005, 0.0, 1.0)  # split_shrink 0
    m = B.gs_map(p, p, p, p, p, 10, 3)
    empty = B.gs_map(p, p, p, p, p, 0, 3)
    assert lib.gs_densify_count(ctypes.byref(m), p, p, ctypes.byref(badcfg), p, p, None) == \
        B.GS_ERR_INVALID
    assert lib.gs_densify_count(ctypes.byref(empty), p, p, ctypes.byref(good), p, p, None) == \
        B.GS_ERR_INVALID
    g = B.gs_map_grad(p, p, p, p, p)
    nullg = B.gs_map_grad(None, p, p, p, p)
    assert lib.gs_densify_apply(ctypes.byref(m), ctypes.byref(g), ctypes.byref(g), p, p, p,
                                ctypes.byref(good), p, 10, ctypes.byref(nullg), ctypes.byref(g),
                                ctypes.byref(g), p, None) == B.GS_ERR_INVALID
    assert lib.gs_densify_apply(ctypes.byref(m), ctypes.byref(g), ctypes.byref(g), p, p, p,
                                ctypes.byref(good), p, -1, ctypes.byref(g), ctypes.byref(g),
                                ctypes.byref(g), p, None) == B.GS_ERR_INVALID


def test_param_layout_alignment():
    for n, deg in [(1, 0), (3, 3), (1000, 3), (777, 1)]:
        off, total = mapping.param_layout(n, deg)
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            assert off[k] % 64 == 0
        assert off["sh_rest"] == off["sh"] + 3 * n
        assert total >= off["sh"] + 3 * (deg + 1) ** 2 * n and total % 64 == 0

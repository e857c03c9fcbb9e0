"""GPU parity of the point-cloud densification (paper Sec. III-A) against
the FP64 oracle.

Bars: selections exact on images whose values are multiples of 2^-10 (the
squared gradients are then exact in FP32, so both sides take the same
decisions) with thresholds of the same kind; interpolated depths within
1e-6 relative (an FP32 mean of three values) on a triangulation given to
both sides; the full keyframe pipeline on a ray-cast image producing depths
within the range of its vertices' depths.
"""
import numpy as np
import pytest
import torch
from scipy.spatial import Delaunay

import oracle
from paper_2409_13055_gb300 import binding as B
from paper_2409_13055_gb300 import pointcloud, scenes

pytestmark = pytest.mark.gpu

THR = (2.0 ** -8, 2.0 ** -10, 2.0 ** -12)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_13055_gb300 import build
    build.build()
    B.lib()


def _image(H, W, seed):
    rng = np.random.default_rng(seed)
    # smooth-ish field with edges, quantised to multiples of 2^-10
    y, x = np.mgrid[0:H, 0:W]
    f = 0.5 + 0.2 * np.sin(x / 7.0) * np.cos(y / 5.0) + 0.2 * (rng.uniform(size=(H, W)) < 0.02)
    f[:, W // 3:W // 3 + 2] = 0.0
    f = np.round(np.clip(f, 0, 1) * 1024) / 1024
    # a weak 48x48 ramp (slope 20/1024): too flat for the first two passes,
    # so its inner 16x16 block is left to the third
    r0, c0 = (0, 32) if H < 100 else (224, 400)
    f[r0:r0 + 48, c0:c0 + 48] = (307 + 20 * np.arange(48))[None, :] / 1024.0
    return f


@pytest.mark.parametrize("H,W", [(61, 83), (480, 752)])
def test_selection_matches_oracle(H, W):
    img = _image(H, W, H)
    g2, sel = pointcloud.select_pixels(torch.tensor(img, dtype=torch.float32, device="cuda"), 4,
                                       THR)
    want = oracle.select_pixels(img, 4, THR)
    np.testing.assert_array_equal(g2.cpu().numpy(), oracle.grad_sq(img).astype(np.float32))
    np.testing.assert_array_equal(sel.cpu().numpy(), want)
    assert all(np.any(want == k + 1) for k in range(3))


def test_interpolation_matches_oracle_on_a_given_triangulation():
    H, W = 90, 120
    img = _image(H, W, 5)
    sel = oracle.select_pixels(img, 4, THR)
    ys, xs = np.nonzero(sel)
    xy = np.stack([xs, ys], 1)
    tri = Delaunay(xy.astype(float)).simplices.astype(np.int32)
    # counter-clockwise, as both sides require
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cw = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]) < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    depth = np.random.default_rng(6).uniform(1.0, 4.0, len(xy)).astype(np.float32)
    want = oracle.interp_depth(tri, xy, depth.astype(np.float64), img, sel, 4, 2.0 ** -12)
    dev = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    g2 = dev(oracle.grad_sq(img), torch.float32)
    got = pointcloud.interpolate(dev(tri, torch.int32), dev(xy, torch.int32),
                                 dev(depth, torch.float32), g2, dev(sel, torch.int32), 4,
                                 2.0 ** -12).cpu().numpy()
    assert np.count_nonzero(want) > 50
    np.testing.assert_array_equal(got != 0, want != 0)
    np.testing.assert_allclose(got, want, rtol=1e-6)


def test_keyframe_pipeline_on_a_ray_cast_image():
    view = scenes.drone_loop(4, width=188, height=120, f=115.0)[1]
    faces, tex = scenes.room_textures()
    depth, gray = scenes.ray_cast(view, faces, tex)
    D = torch.tensor(depth, device="cuda")
    G = torch.tensor(gray, device="cuda")
    px, py, z = pointcloud.keyframe_points(G, lambda x, y: D[y, x], grid=4,
                                           flat_sq=pointcloud.DEFAULT_THRESHOLDS_SQ[-1])
    n_sel = int(torch.count_nonzero(pointcloud.select_pixels(G)[1]).item())
    assert px.numel() > n_sel > 20  # the interpolation adds points
    assert float(z.min()) >= float(D.min()) - 1e-4 and float(z.max()) <= float(D.max()) + 1e-4
    new = pointcloud.gaussians_from_points(view, px, py, z, G)
    assert new["means"].shape == (px.numel(), 3) and np.all(np.isfinite(new["means"]))

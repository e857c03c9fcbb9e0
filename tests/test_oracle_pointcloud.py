"""Pins of the oracle's point-cloud densification (paper Sec. III-A:
DSO-style pixel selection, Delaunay mean-depth interpolation).

References used: the gradient of a linear ramp (exact), hand-built images
with known per-block winners and a later pass filling an empty region,
explicit first-in-raster-order ties, and the interpolation of one triangle
pair checked pixel by pixel against barycentric containment.
"""
import numpy as np

import oracle


def test_gradient_of_a_ramp_and_the_border():
    y, x = np.mgrid[0:8, 0:10].astype(float)
    g2 = oracle.grad_sq(0.1 * x + 0.2 * y)
    assert np.allclose(g2[1:-1, 1:-1], 0.01 + 0.04)
    assert np.all(g2[0] == 0) and np.all(g2[:, 0] == 0) and np.all(g2[-1] == 0)


def test_selection_per_block_passes_and_ties():
    img = np.zeros((16, 16))
    img[5, 2] = 1.0      # gradient at its neighbours (5,1), (5,3), (4,2), (6,2)
    img[10, 12] = 0.5
    sel = oracle.select_pixels(img, 4, [0.01, 0.0001])
    # block (4..8, 0..4): the ties (5,1), (5,3), (4,2), (6,2) -> first in raster order (4,2)
    assert sel[4, 2] == 1
    assert sel[9, 12] == 1 or sel[10, 11] == 1 or sel[10, 13] == 1 or sel[11, 12] == 1
    # pass 2 on 8x8 blocks: only blocks without any pass-1 pixel; the image is
    # flat there, so nothing reaches the threshold
    assert np.count_nonzero(sel == 2) == 0
    # a weak edge in an empty 8x8 block is picked by the second pass only
    img2 = img.copy()
    img2[2, 12] = 0.03
    sel2 = oracle.select_pixels(img2, 4, [0.01, 0.0001])
    assert np.count_nonzero(sel2[0:8, 8:16] == 1) == 0
    assert np.count_nonzero(sel2[0:8, 8:16] == 2) == 1


def test_interpolation_mean_of_vertices_on_flat_pixels():
    xy = np.array([[0, 0], [12, 0], [0, 12], [12, 12]])
    depth = np.array([1.0, 2.0, 4.0, 8.0])
    tri = np.array([[0, 1, 2], [1, 3, 2]])
    gray = np.zeros((13, 13))
    sel = np.zeros((13, 13), np.int32)
    out = oracle.interp_depth(tri, xy, depth, gray, sel, 3, 1e-6)
    for gy in range(5):
        for gx in range(5):
            x, y = 3 * gx, 3 * gy
            want = (1 + 2 + 4) / 3 if x + y <= 12 else (2 + 8 + 4) / 3
            assert abs(out[gy, gx] - want) < 1e-12, (x, y)
    sel[0, 0] = 1
    assert oracle.interp_depth(tri, xy, depth, gray, sel, 3, 1e-6)[0, 0] == 0

"""The host Delaunay triangulation of tracked pixels (paper Sec. III-A,
gs_delaunay), against scipy (Qhull) where the triangulation is unique and,
on integer grids full of co-circular points, against the defining
properties: counter-clockwise non-degenerate triangles, no point strictly
inside any circumcircle (exact integer arithmetic), 2n - h - 2 triangles,
and a union of area equal to the convex hull's."""
import numpy as np
import pytest
from scipy.spatial import ConvexHull, Delaunay

from paper_2409_13055_gb300 import binding as B


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2409_13055_gb300 import build
    build.build()
    B.lib()


def _orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def _check_valid(pts, tri):
    P = [tuple(int(v) for v in p) for p in pts]
    n = len(P)
    area2 = 0
    for t in tri:
        a, b, c = (P[i] for i in t)
        o = _orient(a, b, c)
        assert o > 0
        area2 += o
        ax, ay, bx, by, cx, cy = a[0], a[1], b[0], b[1], c[0], c[1]
        for d in P:
            adx, ady, bdx, bdy, cdx, cdy = ax - d[0], ay - d[1], bx - d[0], by - d[1], cx - d[0], cy - d[1]
            det = (adx * (bdy * (cdx * cdx + cdy * cdy) - cdy * (bdx * bdx + bdy * bdy))
                   - ady * (bdx * (cdx * cdx + cdy * cdy) - cdx * (bdx * bdx + bdy * bdy))
                   + (adx * adx + ady * ady) * (bdx * cdy - cdx * bdy))
            assert det <= 0, (t, d)
    hull = ConvexHull(np.asarray(pts, float))
    assert abs(area2 / 2 - hull.volume) < 1e-6
    # points on the hull boundary, collinear ones included
    hv = np.asarray(pts, float)[hull.vertices]
    on = 0
    for p in np.asarray(pts, float):
        for i in range(len(hv)):
            a, b = hv[i], hv[(i + 1) % len(hv)]
            if abs((b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])) < 1e-9 and \
                    min(a[0], b[0]) - 1e-9 <= p[0] <= max(a[0], b[0]) + 1e-9 and \
                    min(a[1], b[1]) - 1e-9 <= p[1] <= max(a[1], b[1]) + 1e-9:
                on += 1
                break
    assert len(tri) == 2 * n - on - 2


@pytest.mark.parametrize("n", [3, 50, 3000])
def test_matches_scipy_in_general_position(n):
    rng = np.random.default_rng(n)
    pts = np.unique(rng.integers(0, 1 << 19, size=(n, 2)), axis=0)
    tri = B.gs_delaunay(pts)
    want = Delaunay(pts.astype(float)).simplices
    assert set(tuple(sorted(t)) for t in tri.tolist()) == set(tuple(sorted(t)) for t in want.tolist())


def test_integer_grid_of_cocircular_points_is_a_valid_delaunay_triangulation():
    ys, xs = np.mgrid[0:10, 0:10]
    pts = np.stack([xs.ravel() * 3, ys.ravel() * 2], 1)
    _check_valid(pts, B.gs_delaunay(pts))


def test_random_pixels_of_a_small_image():
    rng = np.random.default_rng(7)
    flat = rng.choice(64 * 48, size=400, replace=False)
    pts = np.stack([flat % 64, flat // 64], 1)
    _check_valid(pts, B.gs_delaunay(pts))


def test_degenerate_inputs():
    assert B.gs_delaunay(np.array([[0, 0], [5, 5], [9, 9], [2, 2]])).shape == (0, 3)
    assert B.gs_delaunay(np.array([[0, 0], [1, 0]])).shape == (0, 3)
    with pytest.raises(B.GSError):
        B.gs_delaunay(np.array([[0, 0], [1, 0], [0, 0], [0, 1]]))

"""Pins of the oracle's projection step (Sec. II: projecting Gaussians onto the
camera plane; Sec. III-B: the original 3DGS rasteriser).

Each check compares against something the oracle does not compute itself:
textbook pinhole projection, closed forms for isotropic and axis-aligned
Gaussians, the rotation convention of a known quaternion, rigid-motion
invariance, scipy's spherical harmonics, and central finite differences.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from paper_2409_13055_gb300 import scenes


def one_gaussian(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, sh=None, degree=0):
    K = (degree + 1) ** 2
    shv = np.zeros((K, 1, 3)) if sh is None else np.asarray(sh, float).reshape(K, 1, 3)
    return dict(means=np.array([mean], float), log_scales=np.array([log_scale], float),
                quats=np.array([quat], float), opacity_logits=np.array([logit], float),
                sh=shv, sh_degree=degree)


# ----------------------------------------------------------------------------
# Spherical harmonics against scipy.
# ----------------------------------------------------------------------------
def real_sh_scipy(l, m, d):
    """Real SH with the Condon-Shortley phase from scipy's complex Y_l^m."""
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        return special.sph_harm_y(l, 0, theta, phi).real
    if m > 0:
        return math.sqrt(2) * special.sph_harm_y(l, m, theta, phi).real
    return math.sqrt(2) * special.sph_harm_y(l, -m, theta, phi).imag


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        got = oracle.sh_basis(3, d)
        want = [real_sh_scipy(l, m, d) for l in range(4) for m in range(-l, l + 1)]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------
# Pinhole projection of the mean, textbook form.
# ----------------------------------------------------------------------------
def test_mean_projection_is_pinhole():
    rng = np.random.default_rng(1)
    R, t = scenes.random_pose(rng, 0.5, 20.0)
    view = scenes.camera(640, 480, 525.0, 520.0, 318.0, 242.0, R=R, t=t)
    pts = rng.uniform(-0.5, 0.5, (50, 3)) + np.array([0, 0, 2.5])
    p = dict(means=pts, log_scales=np.full((50, 3), -4.0), quats=np.tile([1.0, 0, 0, 0], (50, 1)),
             opacity_logits=np.zeros(50), sh=np.zeros((1, 50, 3)), sh_degree=0)
    pr = oracle.project(p, view)
    Kmat = np.array([[525.0, 0, 318.0], [0, 520.0, 242.0], [0, 0, 1]])
    Xc = (R.astype(float) @ pts.T).T + t.astype(float)
    uvw = (Kmat @ Xc.T).T
    vis = pr["tiles_touched"] > 0
    assert vis.sum() > 30
    np.testing.assert_allclose(pr["mean2d"][vis], (uvw[:, :2] / uvw[:, 2:])[vis], rtol=1e-13)
    np.testing.assert_allclose(pr["depth"], Xc[:, 2], rtol=1e-14)


# ----------------------------------------------------------------------------
# Isotropic Gaussian on the optical axis: Sigma' = ((f s / z)^2 + 0.3) I.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("z,log_s,f", [(2.0, -4.0, 300.0), (1.0, -3.0, 525.0), (3.7, -5.0, 600.0)])
def test_isotropic_on_axis_closed_form(z, log_s, f):
    W, H = 320, 240
    view = scenes.camera(W, H, f, f)
    pr = oracle.project(one_gaussian([0, 0, z], [log_s] * 3, logit=0.3), view, tight=False)
    s = math.exp(log_s)
    var = (f * s / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [var, 0.0, var], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(pr["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(pr["mean2d"][0], [W / 2, H / 2], rtol=1e-15)
    r = math.ceil(3 * math.sqrt(var))
    assert pr["radius"][0] == r
    x0, y0 = math.floor((W / 2 - r) / 16), math.floor((H / 2 - r) / 16)
    x1, y1 = math.floor((W / 2 + r + 15) / 16), math.floor((H / 2 + r + 15) / 16)
    assert list(pr["rect"][0]) == [max(0, x0), max(0, y0), min(20, x1), min(15, y1)]
    assert pr["tiles_touched"][0] == (min(20, x1) - max(0, x0)) * (min(15, y1) - max(0, y0))
    np.testing.assert_allclose(pr["opacity"][0], 1 / (1 + math.exp(-0.3)), rtol=1e-15)


def test_isotropic_off_axis_closed_form():
    """Isotropic Sigma = s^2 I: Sigma' = s^2 J J^T + 0.3 I with J of the pinhole."""
    f, z, x, y, s = 400.0, 2.0, 0.3, -0.2, 0.02
    view = scenes.camera(640, 480, f, f)
    pr = oracle.project(one_gaussian([x, y, z], [math.log(s)] * 3), view)
    J = np.array([[f / z, 0, -f * x / z ** 2], [0, f / z, -f * y / z ** 2]])
    C = s * s * J @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(pr["cov2d"][0], [C[0, 0], C[0, 1], C[1, 1]], rtol=1e-12)


def test_quaternion_convention_rotates_axes_actively():
    """q = (cos 22.5deg, 0, 0, sin 22.5deg) turns the local x axis towards +y:
    Sigma_xy = (s1^2 - s2^2)/2 > 0 for s1 > s2 (a transposed rotation flips the sign)."""
    f, z = 500.0, 2.0
    s1, s2, s3 = 0.05, 0.01, 0.02
    th = math.radians(45)
    q = (math.cos(th / 2), 0, 0, math.sin(th / 2))
    view = scenes.camera(640, 480, f, f)
    pr = oracle.project(one_gaussian([0, 0, z], [math.log(s1), math.log(s2), math.log(s3)], q), view)
    k = (f / z) ** 2
    a, b = s1 * s1, s2 * s2
    want = [k * (a + b) / 2 + 0.3, k * (a - b) / 2, k * (a + b) / 2 + 0.3]
    np.testing.assert_allclose(pr["cov2d"][0], want, rtol=1e-12)


def test_quaternion_sign_and_scale_invariance():
    p, view = scenes.tiny_scene(40, 64, 48, seed=5)
    base = oracle.project(p, view)
    for fac in (-1.0, 2.5):
        q = dict(p)
        q["quats"] = p["quats"].astype(float) * fac
        other = oracle.project(q, view)
        np.testing.assert_allclose(other["cov2d"], base["cov2d"], rtol=1e-12, atol=1e-12)


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_rigid_motion_invariance():
    """Moving the map by a rigid motion G and the camera with it changes nothing
    on screen: mean2d, depth and cov2d are invariant (SH degree 0)."""
    p, view = scenes.tiny_scene(50, 96, 64, seed=6)
    base = oracle.project(p, view)
    ang = 0.7
    ax = np.array([0.3, -0.5, 0.8])
    ax /= np.linalg.norm(ax)
    qg = np.array([math.cos(ang / 2), *(math.sin(ang / 2) * ax)])
    Rg = scenes._rotation_from_axis_angle(ax, ang)
    tg = np.array([0.4, -1.0, 2.0])
    moved = dict(p)
    moved["means"] = (Rg @ p["means"].astype(float).T).T + tg
    moved["quats"] = np.stack([quat_mul(qg, q) for q in p["quats"].astype(float)])
    v2 = dict(view)
    R = np.asarray(view["R"], float)
    v2["R"] = R @ Rg.T
    v2["t"] = np.asarray(view["t"], float) - R @ Rg.T @ tg
    other = oracle.project(moved, v2)
    np.testing.assert_allclose(other["mean2d"], base["mean2d"], rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(other["depth"], base["depth"], rtol=1e-12)
    np.testing.assert_allclose(other["cov2d"], base["cov2d"], rtol=1e-10, atol=1e-10)


def test_culling_near_plane_and_nonfinite():
    view = scenes.camera(64, 48, 64.0, 64.0)
    p = one_gaussian([0, 0, 0.1], [-4] * 3)
    assert oracle.project(p, view)["tiles_touched"][0] == 0
    p = one_gaussian([0, 0, -1.0], [-4] * 3)
    assert oracle.project(p, view)["tiles_touched"][0] == 0
    p = one_gaussian([0, 0, float("nan")], [-4] * 3)
    assert oracle.project(p, view)["tiles_touched"][0] == 0
    p = one_gaussian([0, 0, 1.0], [float("inf")] * 3)
    assert oracle.project(p, view)["tiles_touched"][0] == 0
    p = one_gaussian([50.0, 0, 1.0], [-4] * 3)  # far outside the image: empty rect
    assert oracle.project(p, view)["tiles_touched"][0] == 0


def test_sh_degree0_colour_and_clamp():
    view = scenes.camera(64, 48, 64.0, 64.0)
    y00 = 0.5 / math.sqrt(math.pi)
    p = one_gaussian([0, 0, 1.0], [-4] * 3, sh=[[0.2 / y00, -0.7 / y00, 0.0]])
    pr = oracle.project(p, view)
    np.testing.assert_allclose(pr["rgb"][0], [0.7, 0.0, 0.5], atol=1e-15)
    assert list(pr["clamped"][0]) == [0, 1, 0]


def test_sh_colour_uses_direction_from_camera_centre():
    """Degree-1 colour = 0.5 + sum_k Y_k(dir) c_k with dir from the camera centre."""
    rng = np.random.default_rng(3)
    R, t = scenes.random_pose(rng, 0.5, 25.0)
    view = scenes.camera(128, 96, 100.0, 100.0, R=R, t=t)
    center = -R.astype(float).T @ t.astype(float)
    mean = center + (R.astype(float).T @ np.array([0.05, -0.02, 1.5]))
    sh = rng.normal(0, 0.2, (4, 1, 3))
    pr = oracle.project(one_gaussian(mean, [-4] * 3, sh=sh, degree=1), view)
    d = mean - center
    d /= np.linalg.norm(d)
    Y = [real_sh_scipy(l, m, d) for l in range(2) for m in range(-l, l + 1)]
    want = np.maximum(0.0, 0.5 + np.einsum("k,kc->c", Y, sh[:, 0, :]))
    np.testing.assert_allclose(pr["rgb"][0], want, rtol=1e-12)


# ----------------------------------------------------------------------------
# Projection adjoint against central finite differences (h = 1e-6).
# ----------------------------------------------------------------------------
def _proj_scalar(params, view, w):
    pr = oracle.project(params, view)
    return (np.sum(w["dmean2d"] * pr["mean2d"]) + np.sum(w["dconic"] * pr["conic"]) +
            np.sum(w["dopacity"] * pr["opacity"]) + np.sum(w["drgb"] * pr["rgb"])), pr


@pytest.mark.parametrize("degree,offscreen", [(0, False), (3, False), (3, True)])
def test_project_bwd_matches_central_differences(degree, offscreen):
    rng = np.random.default_rng(10 + degree + 5 * offscreen)
    n = 12
    p, view = scenes.tiny_scene(n, 64, 48, seed=20 + degree, sh_degree=degree)
    p = {k: (v.astype(float) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    R, t = scenes.random_pose(rng, 0.3, 15.0)
    view["R"], view["t"] = R.astype(float), t.astype(float) * 0.2
    if offscreen:  # push some means sideways so the Jacobian clamp engages
        p["means"][: n // 2, 0] += 1.6 * p["means"][: n // 2, 2]
    w = dict(dmean2d=rng.normal(size=(n, 2)), dconic=rng.normal(size=(n, 3)),
             dopacity=rng.normal(size=n), drgb=rng.normal(size=(n, 3)))
    base_val, pr = _proj_scalar(p, view, w)
    vis = pr["tiles_touched"] > 0
    assert vis.sum() >= n // 3
    for k in w:  # culled Gaussians take no part in the render and get no gradient
        w[k][~vis] = 0.0
    g = oracle.project_bwd(p, view, w)
    h = 1e-6
    checked = 0
    for key in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = p[key]
        flat = arr.reshape(-1)
        gflat = g[key].reshape(-1)
        for j in range(flat.size):
            old = flat[j]
            flat[j] = old + h
            fp, prp = _proj_scalar(p, view, w)
            flat[j] = old - h
            fm, prm = _proj_scalar(p, view, w)
            flat[j] = old
            if not (np.array_equal(prp["clamped"], prm["clamped"]) and
                    np.array_equal(prp["tiles_touched"] > 0, prm["tiles_touched"] > 0)):
                continue
            fd = (fp - fm) / (2 * h)
            assert abs(fd - gflat[j]) <= 1e-5 * max(1.0, abs(fd)), (key, j, fd, gflat[j])
            checked += 1
    assert checked > 0.9 * sum(p[k].size for k in ("means", "log_scales", "quats",
                                                         "opacity_logits", "sh"))


# ----------------------------------------------------------------------------
# Tight rects (reading C19): the square rect cut to the box of the ellipse
# outside which alpha = o exp(-q/2) < 1/255, widened to q <= 1.01 t + 0.01.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("z,log_s,f,logit", [(2.0, -4.0, 300.0, 0.3), (1.0, -3.0, 525.0, -2.0),
                                             (3.7, -4.5, 600.0, -4.5), (1.5, -3.5, 400.0, 3.0)])
def test_tight_rect_isotropic_closed_form(z, log_s, f, logit):
    W, H = 320, 240
    view = scenes.camera(W, H, f, f)
    pr = oracle.project(one_gaussian([0, 0, z], [log_s] * 3, logit=logit), view, tight=True)
    var = (f * math.exp(log_s) / z) ** 2 + 0.3
    o = 1 / (1 + math.exp(-logit))
    r = math.ceil(3 * math.sqrt(var))
    sq = [max(0, math.floor((W / 2 - r) / 16)), max(0, math.floor((H / 2 - r) / 16)),
          min(20, math.floor((W / 2 + r + 15) / 16)), min(15, math.floor((H / 2 + r + 15) / 16))]
    h = math.sqrt((1.01 * 2 * math.log(255 * o) + 0.01) * var)
    box = [math.ceil((W / 2 - h - 15) / 16), math.ceil((H / 2 - h - 15) / 16),
           math.floor((W / 2 + h) / 16) + 1, math.floor((H / 2 + h) / 16) + 1]
    want = [max(sq[0], box[0]), max(sq[1], box[1]), min(sq[2], box[2]), min(sq[3], box[3])]
    assert list(pr["rect"][0]) == want
    # the tiles of the box whose pixel square comes within h of the centre
    # (a circle here: distance from the centre to the tile's pixel rectangle)
    cx, cy = W / 2, H / 2
    n = 0
    for ty in range(want[1], want[3]):
        for tx in range(want[0], want[2]):
            ddx = max(tx * 16 - cx, 0.0, cx - (tx * 16 + 15))
            ddy = max(ty * 16 - cy, 0.0, cy - (ty * 16 + 15))
            n += ddx * ddx + ddy * ddy <= h * h
    assert pr["tiles_touched"][0] == n


def test_tight_rect_empty_below_alpha_threshold():
    """o < 0.999/255: alpha < 1/255 at every pixel, so no tile at all."""
    view = scenes.camera(320, 240, 300.0, 300.0)
    logit = math.log((0.99 / 255) / (1 - 0.99 / 255))
    pr = oracle.project(one_gaussian([0, 0, 2.0], [-3.0] * 3, logit=logit), view, tight=True)
    assert pr["tiles_touched"][0] == 0
    assert oracle.project(one_gaussian([0, 0, 2.0], [-3.0] * 3, logit=logit), view,
                          tight=False)["tiles_touched"][0] > 0


def _min_q_over_rect(a, b, c, x0, x1, y0, y1):
    """min of q = a x^2 + 2 b x y + c y^2 over the rectangle [x0,x1] x [y0,y1]
    (coordinates relative to the centre; a, c > 0, ac > b^2)."""
    if x0 <= 0 <= x1 and y0 <= 0 <= y1:
        return 0.0
    best = np.inf
    for x in (x0, x1):  # vertical edges: minimise over y in [y0, y1]
        y = min(max(-b * x / c, y0), y1)
        best = min(best, a * x * x + 2 * b * x * y + c * y * y)
    for y in (y0, y1):
        x = min(max(-b * y / a, x0), x1)
        best = min(best, a * x * x + 2 * b * x * y + c * y * y)
    return best


@pytest.mark.parametrize("tile,large", [((16, 16), False), ((8, 8), False), ((8, 8), True)])
def test_tight_tiles_are_exactly_those_meeting_the_ellipse(tile, large):
    """Brute force over pixels and tiles: each Gaussian's tight tiles (its
    row spans, read back from the tight binning) are exactly the tiles of
    its square rect whose pixel rectangle meets the widened ellipse
    q <= 1.01 * 2 ln(255 o) + 0.01 (q in the conic), which holds every
    pixel with alpha >= 1/255; every other tile of the square rect has alpha
    < 1/255 at all its pixels.  The set is geometric for every box shape:
    the large case holds boxes of one tile row, of one tile column and of
    more than 16 tile rows."""
    tw, th = tile
    W, H = (320, 240) if large else (160, 120)
    rng = np.random.default_rng(6 if large else 5)
    R, t = scenes.random_pose(rng, 0.3, 20.0)
    view = scenes.camera(W, H, 150.0, 150.0, R=R, t=t)
    n = 300
    q = rng.normal(size=(n, 4))
    ls = rng.normal(-3.5, 0.8, (n, 3))
    if large:  # a third of them large, the rest small enough for one-row boxes
        ls = np.where(np.arange(n)[:, None] < n // 3, rng.normal(-2.2, 0.9, (n, 3)),
                      rng.normal(-4.5, 0.8, (n, 3)))
    p = dict(means=rng.uniform(-0.6, 0.6, (n, 3)) + np.array([0, 0, 2.0]),
             log_scales=ls, quats=q / np.linalg.norm(q, axis=1)[:, None],
             opacity_logits=rng.normal(-1.0, 2.0, n), sh=np.zeros((1, n, 3)), sh_degree=0)
    sq = oracle.project(p, view, tw, th, tight=False)
    ti = oracle.project(p, view, tw, th, tight=True)
    tx_n, ty_n = oracle.tile_grid(W, H, tw, th)
    start, lst = oracle.bin_tiles(ti["depth"].astype(np.float32), ti["rect"], ti["tiles_touched"],
                                  tx_n, ty_n, ti, tile)
    tiles_of = [set() for _ in range(n)]
    for tile_id in range(tx_n * ty_n):
        for g in lst[start[tile_id]:start[tile_id + 1]]:
            tiles_of[g].add(tile_id)
    ys, xs = np.mgrid[0:H, 0:W]
    dropped = kept = 0
    for i in np.flatnonzero(sq["tiles_touched"] > 0):
        a, b, c = sq["conic"][i]
        mx, my = sq["mean2d"][i]
        o = sq["opacity"][i]
        dx, dy = xs - mx, ys - my
        alpha = np.minimum(0.99, o * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy))
        lvl = 1.01 * 2 * np.log(255 * o) + 0.01 if 255 * o >= 0.999 else -1.0
        s0 = sq["rect"][i]
        assert len(tiles_of[i]) == ti["tiles_touched"][i]
        for ty in range(s0[1], s0[3]):
            for tx in range(s0[0], s0[2]):
                inside = ty * tx_n + tx in tiles_of[i]
                qmin = _min_q_over_rect(a, b, c, tx * tw - mx, tx * tw + tw - 1 - mx,
                                        ty * th - my, ty * th + th - 1 - my)
                meets = lvl >= 0 and qmin <= lvl
                if ti["guard"][i] & oracle.GUARD_TIGHT == 0 and abs(qmin - lvl) > 1e-9 * (1 + lvl):
                    assert inside == meets, (i, tx, ty, qmin, lvl)
                if not inside:
                    dropped += 1
                    blk = alpha[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw]
                    assert blk.max() < 1 / 255, (i, tx, ty, blk.max())
                else:
                    kept += 1
    assert dropped > 50 and kept > 50  # the cut is not vacuous on this scene
    if large:
        vis = ti["tiles_touched"] > 0
        rows = (ti["rect"][:, 3] - ti["rect"][:, 1])[vis]
        cols = (ti["rect"][:, 2] - ti["rect"][:, 0])[vis]
        assert (rows > 16).sum() >= 3 and (rows == 1).sum() >= 3 and (cols == 1).sum() >= 3, (
            (rows > 16).sum(), (rows == 1).sum(), (cols == 1).sum())

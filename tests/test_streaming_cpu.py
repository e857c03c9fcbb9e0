"""Host-side checks of the streaming workload: the keyframe generator (loop
geometry, analytic ray cast, DSO-like point selection) and the map's
insertion (GaussianMap.append on CPU tensors)."""
import numpy as np
import torch

from paper_2409_13055_gb300 import mapping, scenes


def _centre(v):
    return -np.asarray(v["R"], np.float64).T @ np.asarray(v["t"], np.float64)


def test_drone_loop_is_a_closed_5m_loop():
    views = scenes.drone_loop(50, jitter_m=0.0, jitter_deg=0.0)
    c = np.stack([_centre(v) for v in views])[:, [0, 2]]  # the horizontal loop
    steps = np.linalg.norm(np.diff(np.vstack([c, c[:1]]), axis=0), axis=1)
    # 50 equal chords of a circle of circumference 5: 5 sin(pi/50) / (pi/50)
    want = 5.0 * np.sin(np.pi / 50) / (np.pi / 50)
    np.testing.assert_allclose(steps, want / 50, rtol=1e-5)  # poses are float32
    for v in views:
        R = np.asarray(v["R"], np.float64)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
        assert v["channels"] == 1 and (v["width"], v["height"]) == (752, 480)


def test_ray_cast_hits_the_wall_at_its_distance():
    """A camera at (0, 0, 0.5) looking down +z sees, on rows at and above
    the horizon (the boxes stand below y = 0.5), the far wall z = 5 at depth
    4.5 with the wall's texture formula, and the side walls x = +-3 at depth
    3 / |x_n| towards the image edges."""
    faces, tex = scenes.room_textures()
    far = [i for i, (O, U, V) in enumerate(faces[:6]) if abs(O[2] - 5.0) < 1e-9 and U[2] == 0
           and V[2] == 0][0]
    view = scenes.camera(64, 48, 40.0, 40.0, t=np.array([0.0, 0.0, -0.5], np.float32))
    depth, gray = scenes.ray_cast(view, faces, tex)
    assert np.all(np.isfinite(depth))
    O, U, V = (np.asarray(a, np.float64) for a in faces[far])
    base, amp, per = tex[far]
    xn = (np.arange(64) - 32) / 40.0
    wall = np.abs(xn) * 4.5 < 3.0  # columns that see the far wall; the rest see x = +-3
    for row in (18, 24):
        want_depth = np.where(wall, 4.5, 3.0 / np.maximum(np.abs(xn), 1e-9))
        np.testing.assert_allclose(depth[row], want_depth, rtol=1e-6)
        x = xn * 4.5
        y = (row - 24) / 40.0 * 4.5
        a = (x - O[0]) / U[0]
        b = (y - O[1]) / V[1]
        want = base + amp * np.sin(2 * np.pi * a * abs(U[0]) / per) * \
            np.sin(2 * np.pi * b * abs(V[1]) / per)
        np.testing.assert_allclose(gray[row][wall], want[wall], atol=1e-5)


def test_dso_points_lie_on_the_surfaces():
    """Without depth noise every selected point back-projects onto a face of
    the room (within FP32 rounding), one point per selected block."""
    v = scenes.drone_loop(4, width=188, height=120, f=115.0)[1]
    faces, tex = scenes.room_textures()
    depth, gray = scenes.ray_cast(v, faces, tex)
    new = scenes.dso_points(v, depth, gray, 300, seed=3, block=2, idepth_sigma=0.0)
    X = new["means"].astype(np.float64)
    assert X.shape == (300, 3)
    d = np.full(len(X), np.inf)
    for O, U, V in faces:
        O, U, V = (np.asarray(a, np.float64) for a in (O, U, V))
        n = np.cross(U, V)
        n /= np.linalg.norm(n)
        rel = X - O
        a = rel @ U / (U @ U)
        b = rel @ V / (V @ V)
        inside = (a >= -1e-4) & (a <= 1 + 1e-4) & (b >= -1e-4) & (b <= 1 + 1e-4)
        d = np.where(inside, np.minimum(d, np.abs(rel @ n)), d)
    assert np.max(d) < 1e-4, np.max(d)
    np.testing.assert_array_equal(new["quats"][:, 0], 1.0)
    assert np.all(new["sh"][1:] == 0.0)


def test_map_append_keeps_old_values_and_zeroes_new_moments():
    rng = np.random.default_rng(0)

    def gauss(n):
        return dict(means=rng.normal(size=(n, 3)).astype(np.float32),
                    log_scales=rng.normal(size=(n, 3)).astype(np.float32),
                    quats=rng.normal(size=(n, 4)).astype(np.float32),
                    opacity_logits=rng.normal(size=n).astype(np.float32),
                    sh=rng.normal(size=(16, n, 3)).astype(np.float32), sh_degree=3)

    a, b = gauss(37), gauss(90)
    gm = mapping.GaussianMap(a, device="cpu")
    gm.m.uniform_(1.0, 2.0)
    gm.v.uniform_(1.0, 2.0)
    gm.step.fill_(7)
    m_old = {k: t.clone() for k, t in gm._views(gm.m).items()}
    gm.append(b)
    assert gm.n == gm.capacity == 127
    P = gm.params()
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        np.testing.assert_array_equal(P[k][:37].numpy(), a[k])
        np.testing.assert_array_equal(P[k][37:].numpy(), b[k])
    np.testing.assert_array_equal(P["sh"][:, :37].numpy(), a["sh"])
    np.testing.assert_array_equal(P["sh"][:, 37:].numpy(), b["sh"])
    M = gm._views(gm.m)
    for k in M:
        old = M[k][:, :37] if k == "sh" else M[k][:37]
        new = M[k][:, 37:] if k == "sh" else M[k][37:]
        assert torch.equal(old, m_old[k])
        assert torch.count_nonzero(new) == 0
    assert int(gm.step.item()) == 7
    off, total = mapping.param_layout(127, 3)
    assert gm.total == total and gm.off == off

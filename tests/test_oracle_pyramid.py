"""Pins of the oracle's Gaussian-pyramid level (paper Sec. III-B: targets
smoothed and down-sampled repeatedly).

References used: the impulse response (outer product of the binomial
weights), exactness on constants and on linear ramps away from the border,
the mirrored border by explicit indexing, the output size rule, and the
camera of a level reproducing the projection of the level below at pixel 2i.
"""
import numpy as np

import oracle


def test_impulse_response_is_outer_binomial():
    img = np.zeros((1, 11, 13))
    img[0, 6, 6] = 256.0
    out = oracle.pyr_down(img)
    w = np.array([1, 4, 6, 4, 1], float)
    want = np.zeros((6, 7))
    # output pixel (r, c) samples input (2r, 2c): the kernel centred at 6, 6
    for r in range(6):
        for c in range(7):
            dy, dx = 2 * r - 6, 2 * c - 6
            if abs(dy) <= 2 and abs(dx) <= 2:
                want[r, c] = w[dy + 2] * w[dx + 2]
    np.testing.assert_allclose(out[0], want, atol=1e-12)
    assert out.shape == (1, 6, 7)


def test_constant_and_linear_ramp():
    H, W = 9, 14
    assert np.allclose(oracle.pyr_down(np.full((3, H, W), 0.37)), 0.37, atol=1e-15)
    y, x = np.mgrid[0:H, 0:W].astype(float)
    ramp = (0.2 * x - 0.1 * y + 3.0)[None]
    out = oracle.pyr_down(ramp)
    # interior samples (kernel fully inside) reproduce the ramp at (2r, 2c)
    for r in range(1, (H - 2) // 2):
        for c in range(1, (W - 2) // 2):
            assert abs(out[0, r, c] - (0.2 * 2 * c - 0.1 * 2 * r + 3.0)) < 1e-12


def test_mirrored_border_by_explicit_indexing():
    rng = np.random.default_rng(1)
    img = rng.uniform(size=(2, 5, 6))
    w = np.array([1, 4, 6, 4, 1], float) / 16

    def m(i, n):
        return -i if i < 0 else (2 * n - 2 - i if i >= n else i)

    out = oracle.pyr_down(img)
    for ch in range(2):
        for r in range(3):
            for c in range(3):
                s = 0.0
                for a in range(5):
                    for b in range(5):
                        s += w[a] * w[b] * img[ch, m(2 * r + a - 2, 5), m(2 * c + b - 2, 6)]
                assert abs(out[ch, r, c] - s) < 1e-12


def test_level_camera_maps_pixel_2i_to_i():
    v = dict(width=753, height=481, fx=460.0, fy=455.0, cx=376.2, cy=240.7)
    u = oracle.pyr_view(v)
    assert (u["width"], u["height"]) == (377, 241)
    X = np.array([0.3, -0.2, 2.5])
    px0 = v["fx"] * X[0] / X[2] + v["cx"]
    px1 = u["fx"] * X[0] / X[2] + u["cx"]
    assert abs(px1 - px0 / 2) < 1e-12

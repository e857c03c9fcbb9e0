"""The oracle still reproduces its frozen record (tests/golden/oracle_small.json,
written by tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np

from tests.golden.make_golden import compute

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_frozen_record():
    with open(os.path.join(HERE, "golden", "oracle_small.json")) as f:
        want = json.load(f)
    got = compute()
    assert abs(got["loss"] - want["loss"]) < 1e-12
    assert abs(got["image_sum"] - want["image_sum"]) < 1e-10
    assert abs(got["final_T_sum"] - want["final_T_sum"]) < 1e-10
    assert got["last_idx_sum"] == want["last_idx_sum"]
    np.testing.assert_allclose([p[3] for p in got["pixels"]], [p[3] for p in want["pixels"]],
                               atol=1e-13)
    for k, v in want["grad_norms"].items():
        assert abs(got["grad_norms"][k] - v) <= 1e-10 * max(1.0, abs(v))
    np.testing.assert_allclose(got["grad_means_first"], want["grad_means_first"], rtol=1e-10,
                               atol=1e-15)


def test_tight_rects_change_no_result():
    """Cutting the tile rects to the tiles that can receive alpha >= 1/255
    (reading C19) drops only (Gaussian, tile) pairs that every pixel skips:
    loss, image, transmittance and gradients equal the frozen square-rect
    record; only the list positions (last_idx) move."""
    with open(os.path.join(HERE, "golden", "oracle_small.json")) as f:
        want = json.load(f)
    got = compute(tight=True)
    assert abs(got["loss"] - want["loss"]) < 1e-12
    assert abs(got["image_sum"] - want["image_sum"]) < 1e-10
    assert abs(got["final_T_sum"] - want["final_T_sum"]) < 1e-10
    assert got["last_idx_sum"] <= want["last_idx_sum"]
    np.testing.assert_allclose([p[3] for p in got["pixels"]], [p[3] for p in want["pixels"]],
                               atol=1e-13)
    for k, v in want["grad_norms"].items():
        assert abs(got["grad_norms"][k] - v) <= 1e-10 * max(1.0, abs(v))


def test_threads_change_only_the_last_bits():
    """The oracle's OpenMP loops (used by the benchmark's all-core CPU
    baseline) give the single-threaded results up to the order of additions:
    the frozen record's quantities agree to 1e-12 with four threads."""
    import oracle
    one = compute()
    oracle.set_threads(4)
    try:
        four = compute()
    finally:
        oracle.set_threads(1)
    assert abs(four["loss"] - one["loss"]) < 1e-12
    assert four["last_idx_sum"] == one["last_idx_sum"]
    assert abs(four["image_sum"] - one["image_sum"]) < 1e-12
    for k, v in one["grad_norms"].items():
        assert abs(four["grad_norms"][k] - v) <= 1e-12 * max(1.0, abs(v))

"""Host-side parts of bench.py that need no GPU: the reference arm (the FP64
oracle timed on the host) prints the contract's JSON line, and the
per-iteration roofline adds up its stages."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "room200k_640x480", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "iters/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1
    assert line["config"]["workload"] == "room200k_640x480"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_iteration_roofline_sums_its_stages():
    import bench
    peaks = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "sms": 152}
    n, deg = 1_000_000, 3
    out = bench.iteration_roofline(n, deg, 1, 1200 * 680 * 3, 1200 * 680, 3_000_000,
                                   100_000_000, 12_750, 2, 59 * n, 1.25, peaks)
    stages = out["stages_ms_roof"]
    assert set(stages) == {"project", "bin_sort", "render_fwd", "loss_l1_ssim", "render_bwd",
                           "project_bwd", "adam"}
    assert all(v > 0 for v in stages.values())
    assert out["ms_roof"] == pytest.approx(sum(stages.values()))
    assert out["frac"] == pytest.approx(out["ms_roof"] / 1.25)
    # Adam: 28 B per float of the packed buffer at the copy bandwidth
    assert stages["adam"] == pytest.approx(59 * n * 28 / 6.8e12 * 1e3)
    # the pixel adjoint at 60 FLOP per pair on 152 SMs x 128 lanes x 2 x 2.07 GHz
    assert stages["render_bwd"] == pytest.approx(
        max(100e6 * 60 / (152 * 128 * 2 * 2.07e9), (3e6 * 48 + 1200 * 680 * 16) / 6.8e12) * 1e3)

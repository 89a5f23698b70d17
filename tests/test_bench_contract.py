"""The bench's JSON line: its helpers on the host, and one short run on the GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
gpu = pytest.mark.gpu


def test_profile_traffic_needs_the_kernel_name_and_source_hash():
    """A committed ncu summary supplies the roofline's traffic only for the kernel
    instantiation named on its first line and only while its recorded kernel-source hash
    matches the current sources."""
    import bench
    for tag in ("k_xpass_tma_c64_27q", "k_xpass_wl_c64_27q"):
        path = os.path.join(ROOT, "profiles", tag + ".txt")
        first = open(path).readline()
        name = first.split(" (")[0]
        vals = dict(line.split(":", 1) for line in open(path) if ":" in line and not line.startswith(" "))
        recorded = vals.get("kernel_source_sha256_16", "").strip()
        got = bench.profile_traffic(tag, name)
        if recorded == bench.kernel_source_hash(name):
            assert got is not None and 1e9 < got < 3e9
        else:
            assert got is None
        assert bench.profile_traffic(tag, "k_not_this_kernel") is None


@gpu
def test_bench_line_keeps_its_contract():
    """One short run of the headline leg: a single JSON line with the required keys, the
    dominant kernel's roofline within the measured peak's range and consistent with the
    step time, and end-to-end byte counts."""
    cmd = [sys.executable, "bench.py", "--steps", "4", "--warmup", "3", "--no-cpu", "--no-pergate", "--no-scan",
           "--no-accuracy", "--no-ug32", "--no-protocol", "--adjoint-steps", "0", "--no-autotune"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["steps"] == 4 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["value"] == pytest.approx(4 / (d["ms_per_step"] * 4 / 1000.0), rel=1e-6)
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert 0.3 < rf["frac"] < 1.2 and rf["achieved"] == pytest.approx(rf["frac"] * rf["peak"])
    # the dominant kernel's mean launch fits in the step time it is part of
    assert rf["avg_launch_ms"] * rf["passes_per_step"] / 2 < d["ms_per_step"]
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0 and d["clocks"]["sm_mhz"] > 0

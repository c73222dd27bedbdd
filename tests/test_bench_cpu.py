"""The benchmark's reference arm (the oracle on the host) prints one JSON line
with the fields of the benchmark contract; no GPU is needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "5", "--warmup", "3",
                        "--cpu-seconds", "0.2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert 3 <= d["steps"] <= 5 and d["warmup"] == 3 and d["steps_requested"] == 5
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-6 * d["ms_per_step"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_traffic_reported_only_for_the_captured_x_passes(tmp_path):
    """The bench line's DRAM traffic comes from the committed ncu capture and
    is reported only when the plan runs the x-pass kernels that capture
    measured; the record's total is the sum of its kernels."""
    sys.path.insert(0, ROOT)
    import bench
    tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert tj["matvec_c64_waveguide_bytes"] == sum(tj["kernels"].values())
    x, t = bench.captured_traffic({"x_lines_per_block": 0, "x_lines_per_block_inverse": 0})
    assert x == tj["x_passes"] and t == tj["matvec_c64_waveguide_bytes"]
    assert bench.captured_traffic({"x_lines_per_block": x[0], "x_lines_per_block_inverse": x[1]})[1] == t
    other = {"x_lines_per_block": x[0], "x_lines_per_block_inverse": -x[1]}
    assert bench.captured_traffic(other) == ([x[0], -x[1]], None)
    assert bench.captured_traffic(other, path=str(tmp_path / "absent.json"))[1] is None

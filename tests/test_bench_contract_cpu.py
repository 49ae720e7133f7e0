"""The benchmark's reference arm runs on the host alone: `bench.py --impl reference`
times the CPU oracle on a bounded sample of the QFT30 roundtrip and prints one JSON
line with the keys the benchmark line carries (metric, value, unit, the oracle's
cpu_baseline record, an end-to-end record with no host-device traffic)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["unit"] == "ms" and line["higher_is_better"] is False and line["value"] > 0
    assert line["config"]["workload"] == "qft30_roundtrip" and line["config"]["n_qubits"] == 30
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    # the 30-qubit value is an extrapolation and says so in the line itself; one
    # complete oracle run at a smaller width is measured end to end
    assert line["extrapolated"] is True and cb["extrapolated"] is True
    assert cb["measured_gates"] > 0 and cb["measured_s"] > 0 and cb["scale"] > 1
    full = cb["measured_full_run"]
    assert full["extrapolated"] is False and full["ms"] > 0 and full["error_l2_vs_input"] < 1e-10
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0

"""The reference (oracle) line of bench.py keeps the JSON contract on the host cores (no GPU): one line with
the library line's metric, the oracle as cpu_baseline (a real solve of the workload's right-hand side, its
measured core count, a one-core sample, nothing of the library loaded), and an e2e object without
host-device copies.  Runs the small 48^3 workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line_contract():
    sys.path.insert(0, ROOT)
    import bench
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "lg48",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "RHS/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3 and d["scaling"] == "weak"
    assert d["ms_per_step"] > 0 and d["data"] == "synthetic" and d["dtype"]
    assert d["config"]["workload"] == bench.WORKLOADS["lg48"]["desc"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == "RHS/s" and cb["sample"]
    assert 1 <= cb["cores"] <= (os.cpu_count() or 1)
    assert cb["product_library_loaded"] is False          # the oracle arm loads nothing of the library
    assert cb["solves"] and all(s["converged"] for s in cb["solves"])
    assert cb["one_core"]["cores"] == 1 and cb["one_core"]["s_per_iteration"] > 0
    assert cb["host"]["nproc"] >= 1
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == "RHS/s"
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0

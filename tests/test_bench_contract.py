"""The benchmark's reference arm (the FP64 oracle timed on the host cores) prints one JSON line
with the keys and units of the GPU arm's line; it runs on the CPU, so its contract is checked
here (the GPU arm's line is produced by the same code on a GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    import bench
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "atom-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["scaling"] == "weak" and d["dtype"] == "f64" and d["data"] == "synthetic"
    # value = sample atoms x steps / time and ms_per_step = time / steps: their product is the
    # sample's atom count, which the sample description states
    import re
    n_sample = int(re.search(r"\((\d+) atoms\)", d["cpu_baseline"]["sample"]).group(1))
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - n_sample) < 1e-6 * n_sample
    assert "8000000" in d["config"]["workload"] and d["config"]["n_atoms"] == 8_000_000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

"""The reference arm of bench.py (the FP64 oracle timed on the host cores)
prints the JSON line the benchmark contract asks for, on a small graph."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line(tmp_path):
    out = tmp_path / "ref.json"
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--scale", "12", "--steps", "2",
                          "--warmup", "1", "--out", str(out)], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d == json.loads(out.read_text())
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["higher_is_better"] is True and d["data"] == "synthetic"
    for k in ("metric", "unit", "ms_per_step", "config", "dtype", "scaling"):
        assert k in d
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

"""The reference arm of bench.py (the CPU oracle) prints one JSON line with
the keys of the bench contract; a small grid keeps it to a few seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "16",
                          "--n_t", "4", "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "matvecs/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["grid"] == [16, 16, 16]
    # each step is the sample it times: ms_per_step is the measured sample time
    assert d["ms_per_step"] < d["extrapolated_ms_per_matvec"]


def test_reference_arm_whole_matvec():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--cpu-full",
                          "--n", "16", "--n_t", "4"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                         check=True).stdout
    d = json.loads([ln for ln in out.splitlines() if ln.startswith("{")][0])
    assert d["steps"] == 1 and abs(d["value"] * d["ms_per_step"] / 1000.0 - 1.0) < 1e-9

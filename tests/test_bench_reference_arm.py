"""The benchmark's reference arm (the FP64 oracle on the host cores) on CPU:
one JSON line with the contract's keys, and the instance subset that the
profiling commands use (`--instances`) reaches the line's config."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          *args], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_instance_subset():
    name = "j1j2_L6_J20.6_dh64_ns256"
    d = _line("--instances", name, "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and d["unit"] == "batched steps/s"
    assert d["config"]["instances"] == [name] and d["config"]["n_instances"] == 1
    assert d["value"] > 0 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["dtype"] == "f64"

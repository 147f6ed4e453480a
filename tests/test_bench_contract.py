"""bench.py's output contract, on the CPU.

The reference arm (the FP64 oracle on the host cores) prints one JSON line
with the keys the benchmark contract names; the library's own arm needs a
CUDA device and exits with an error without one (no fallback).
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def has_device():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = run("--impl", "reference", "--workload", "2d64", "--steps", "2", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "GLUPS" and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] >= 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert d["dtype"] == "f64" and d["vs_baseline"] is None
    assert "2+1" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.skipif(has_device(), reason="a CUDA device is present")
def test_own_arm_needs_a_device():
    r = run("--workload", "2d64", "--steps", "1", "--warmup", "3")
    assert r.returncode != 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_traffic_counters_follow_the_kernel_code(tmp_path, monkeypatch):
    """profiles/ncu_traffic.json is valid only for the kernel code it was
    captured on: the hash ignores comments and white space but changes with
    any code token."""
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "paper_1309_3452_gb300" / "csrc"
    src.mkdir(parents=True)
    code = "int f(int a) {\n  return a + 1;  // one more\n}\n/* block */\n"
    for name in bench.KERNEL_SOURCES["step_fp32"]:
        (src / name).write_text(code)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("step_fp32")
    for name in bench.KERNEL_SOURCES["step_fp32"]:
        (src / name).write_text("int f(int a)   {\n\n  return a + 1;  // more than one\n}\n/* another */\n")
    assert bench.kernel_source_hash("step_fp32") == h0
    (src / bench.KERNEL_SOURCES["step_fp32"][0]).write_text(code.replace("+ 1", "+ 2"))
    assert bench.kernel_source_hash("step_fp32") != h0
    # and the committed counters carry the hash of the committed sources
    monkeypatch.setattr(bench, "ROOT", ROOT)
    d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    h = bench.kernel_source_hash("step_fp32")
    assert all(e["source_hash"] == h for k, e in d.items() if k.startswith("step_fp32@"))

"""The reference arm of bench.py (the FP64 oracle timed on the host cores,
one single-threaded process per realisation, all at once): one JSON line with
the benchmark's metric and config on rank 0, nothing on the other ranks.
Runs on the 32^3 GdFeCo workload with two processes so it stays short."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "gdfeco_32",
           "--steps", "2", "--warmup", "1", "--cpu-procs", "2", *args]
    return subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_arm_line():
    out = _run()
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "spin-steps/s" and d["unit"] == "spin-steps/s"
    assert d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0
    assert d["config"]["sample_every"] == 100          # default: once per 100-step chunk
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    c = d["cpu_baseline"]
    assert c["cores"] == 2 and c["nproc"] == os.cpu_count()
    assert c["aggregate"] == d["value"] and 0 < c["per_core"] <= c["aggregate"]
    assert "2 concurrent" in c["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_sampling_option():
    out = _run(None, "--sample-every", "0")
    assert out.returncode == 0, out.stderr
    assert json.loads(out.stdout.strip().splitlines()[-1])["config"]["sample_every"] == 0


def test_reference_arm_other_ranks_silent():
    out = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""

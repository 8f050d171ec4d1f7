"""The benchmark's reference arm (the CPU oracle timed on the host cores) and its JSON contract.

`bench.py --impl reference` needs no GPU: it factors the workload's map with the oracle's banded
LU (Sec. II-C) and substitutes bounded samples of the batch.  Checked here on the 16 x 16 workload:
one JSON line with the fields the driver reads, consistent units and values, and the other ranks
of a multi-process launch exiting without output.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "xbar16_fp64",
           "--steps", "2", "--warmup", "1", *args]
    return subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference"
    assert out["value"] > 0 and out["ms_per_step"] > 0
    assert (out["steps"], out["warmup"]) == (2, 1)
    assert out["higher_is_better"] is True and out["data"] == "synthetic"
    assert out["config"]["workload"] == "xbar16_fp64"
    assert (out["config"]["M"], out["config"]["N"], out["config"]["B"]) == (16, 16, 64)
    cpu = out["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == out["value"] and cpu["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_are_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""

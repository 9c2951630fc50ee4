"""bench.py's reference arm on the host cores (no GPU): one JSON line whose
metric string is the GPU arm's (so the two lines divide), wall time per
step actually spent, the extrapolated trajectory time labelled as a model,
and the keys of the measurement contract; under a multi-rank launch only
rank 0 prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env.setdefault("OMP_NUM_THREADS", "2")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--ref-sample-seconds", "0.2"],
                          capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)


def test_reference_arm_line():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench

    r = _run({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC  # the GPU arm prints the same string
    assert d["unit"] == "s/trajectory" and d["higher_is_better"] is False
    assert d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # the wall time actually spent per step is the sample, not the model
    assert d["ms_per_step"] < 60e3
    assert "model" in d["extrapolated"] and d["extrapolated"]["applications_timed"] >= 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0 and e["value"] == d["value"]
    assert d["config"]["workload"] == bench.WORKLOAD_NAME


def test_reference_arm_other_ranks_print_nothing():
    pytest.importorskip("torch")
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]

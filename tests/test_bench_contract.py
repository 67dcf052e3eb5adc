"""The measurement script's reference arm (the CPU oracle timed on the host
cores) runs without a GPU: its JSON line carries every key of the contract,
and ranks other than 0 exit without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, "bench.py", "--impl", "reference", "--config", "tiny", "--scale", "0.05", "--steps", "2",
       "--warmup", "3", "--cpu-seconds", "1"]


def _run(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_line_has_every_contract_key():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_profiling_query_count_survives_scaling():
    # --queries asks for a number of queries per step whatever --scale does
    sys.path.insert(0, ROOT)
    import bench

    for scale, queries in ((0.05, 123), (0.25, 2000), (0.02, 500)):
        w = bench.make_workload("genome", scale, 16, queries)
        assert len(w.queries) == queries, (scale, queries)
    batches = bench.extra_batches(bench.make_workload("genome", 0.02, 16, 300), 3, 0)
    assert len(batches) == 3 and all(len(b) == 300 for b in batches)
    assert len({hash(b.data.tobytes()) for b in batches}) == 3  # distinct batches of one shape

"""bench.py's reference arm on CPU: the FP64 oracle timed step by step on the host cores,
printed as one JSON line with the same metric, unit and keys as the library's line.

Runs on the plain two-subsystem cell (32^3 grid, 8 bands), whose oracle step takes tens of
milliseconds, so the whole hot path fits every step.  Under several ranks only rank 0 works
and prints; the others exit 0 at once."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, steps=3, warmup=1):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "plain", "--steps", str(steps), "--warmup", str(warmup)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_line_keeps_the_contract():
    lines = _run({"WORLD_SIZE": "1", "RANK": "0", "LOCAL_RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "Embedded H·ψ band-applies/s"
    assert d["unit"] == "band-applies/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    # every step is the whole hot path of the cell: both potentials and all 8 bands
    assert d["config"]["band_applies_per_step"] == 8
    assert abs(d["value"] - 8 / (d["ms_per_step"] / 1e3)) < 1e-9 * d["value"]
    # the timed steps fit inside the arm's own wall clock
    assert d["ms_per_step"] * d["steps"] / 1e3 <= d["wall_s"] * 1.0001
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_only_rank_zero_runs_the_reference_arm():
    assert _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}) == []
    (line,) = _run({"WORLD_SIZE": "2", "RANK": "0", "LOCAL_RANK": "0"}, steps=1, warmup=0)
    assert json.loads(line)["n_gpus"] == 2

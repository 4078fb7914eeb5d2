"""bench.py's reference arm on the host (no GPU): the oracle timed on a
bounded sample, one JSON line with every key of the benchmark contract, and
the non-zero ranks of a multi-rank launch exit without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       cwd=ROOT, env=e, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_line_has_every_key():
    lines = _run("--steps", "2", "--warmup", "1", "--ref-sample", "32")
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "ms_per_step", "dtype", "data"):
        assert d[k]
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["value"] > 0 and d["unit"] == "events/s"
    assert d["config"]["workload"] == "ggttgg_524288" and d["config"]["nevt_per_step"] == 32
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["sample"]
    assert cpu["value"] == d["value"] and cpu["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] * d["value"] / 1e3 - 32) < 1e-6 * 32


def test_nonzero_rank_exits_without_work():
    assert _run("--steps", "1", "--warmup", "0", env={"RANK": "1", "WORLD_SIZE": "2"}) == []

"""The reference arm of bench.py: the FP64 oracle timed on host cores.

It needs no GPU, so the JSON line it prints can be checked here for the keys of
the bench contract, the oracle baseline and the zero-byte end-to-end entry.
"""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *extra],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_line_keeps_the_contract():
    rec = _run("--steps", "1", "--warmup", "3")
    assert rec["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["value"] > 0 and rec["ms_per_step"] > 0
    assert rec["steps"] == 1 and rec["warmup"] == 3 and rec["n_gpus"] == 1
    assert rec["higher_is_better"] is True and rec["vs_baseline"] is None
    assert rec["dtype"] == "f64"
    import bench
    assert rec["config"] == bench._config(bench.BATCH, 1)      # the same config as the GPU arm
    assert rec["sample"] and str(bench.ORACLE_LINES) in rec["sample"]
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["sample"] == rec["sample"]
    assert cb["cpu_model"]
    assert cb["value"] == rec["value"] and cb["unit"] == rec["unit"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_warmup_is_raised_to_three():
    rec = _run("--steps", "1", "--warmup", "0")
    assert rec["warmup"] == 3

"""bench.py's reference arm (the FP64 oracle on the host cores) prints the one
JSON line of the contract: its keys, units and the zero-byte end-to-end entry,
on the default workload (cart-pole 48^4: a bounded sample of level-0 graph
construction per step) and on cstr_256 (one whole oracle solve per step)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", *extra], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "cells/s" and d["value"] > 0
    assert d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    return d


def test_reference_arm_default_workload():
    d = _reference_line()
    assert d["config"]["workload"] == "cartpole_48" and d["config"]["rule"] == "outer"
    assert "level-0 cells" in d["cpu_baseline"]["sample"]
    ph = d["cpu_baseline"]["phases_s"]
    assert set(ph) == {"build_graph"} and ph["build_graph"] * 1e3 == pytest.approx(d["ms_per_step"])


def test_reference_arm_cstr_256():
    d = _reference_line("--workload", "cstr_256")
    assert d["config"]["workload"] == "cstr_256"
    ph = d["cpu_baseline"]["phases_s"]
    assert set(ph) == {"build_graph", "prune", "subdivide"} and all(v >= 0 for v in ph.values())
    assert sum(ph.values()) <= d["ms_per_step"] / 1e3

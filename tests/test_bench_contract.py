"""CPU checks of bench.py's output contract, on its reference arm (the oracle
timed on the host), which needs no GPU: one JSON line with the contract's
keys on rank 0, nothing on the other ranks."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    return [line for line in p.stdout.splitlines() if line.strip()]


@pytest.mark.parametrize("extra", [[], ["--kernel", "bspline"], ["--full-res"]])
def test_reference_arm_json_line(extra):
    lines = _run(["--impl", "reference", "--L", "16", "--J-min", "0", "--steps", "1", "--warmup", "1",
                  "--cpu-orders", "8"] + extra)
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert d["config"]["L"] == 16 and "workload" in d["config"]
    assert d["config"]["multires"] == ("--full-res" not in extra)
    assert d["config"]["kernel"] == ("bspline" if "bspline" in extra else "sd")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    assert _run(["--impl", "reference", "--L", "16", "--J-min", "0", "--steps", "1", "--warmup", "1"],
                env={"RANK": "1", "WORLD_SIZE": "2"}) == []

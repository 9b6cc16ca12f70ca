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


def test_stage_rooflines_follow_the_work_of_each_stage(monkeypatch):
    """The per-stage roofline records on synthetic stage statistics: byte-counted
    stages (ring DFTs, quadrature) against HBM, the Legendre contractions against
    the pipe of their precision, the dominant stage picked by time, and the
    Legendre sub-record always present."""
    import types
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1800.0, "sm_max_mhz": 2000.0}
    steps = 2
    stats = {
        "ring_fwd": dict(launches=4, timed=4, ms=20.0, flops=0.0, bytes=60e9),
        "theta_quad": dict(launches=4, timed=4, ms=30.0, flops=0.0, bytes=12e9),
        "leg_anal": dict(launches=4, timed=4, ms=50.0, flops=1e13, bytes=0.0),
        "leg_synth": dict(launches=4, timed=4, ms=40.0, flops=1e13, bytes=0.0),
        "ring_inv": dict(launches=4, timed=4, ms=20.0, flops=0.0, bytes=60e9),
        "pack": dict(launches=0, timed=0, ms=0.0, flops=0.0, bytes=0.0),
    }
    a = types.SimpleNamespace(steps=steps, precision="tf32x3")
    roof, leg, recs = bench.rooflines(stats, a, peaks, 64, [2048, 8, 4])
    tf32 = 1800.0 * 1.1 / 2.25
    assert roof["kernel"] == "leg_anal" and roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(1e13 / 0.050 / 1e12)
    assert roof["peak"] == pytest.approx(tf32) and roof["frac"] == pytest.approx(200.0 / tf32)
    assert roof["executed_mma_frac"] == pytest.approx(3 * 200.0 / tf32)
    assert "of measured" in roof["peak_source"]
    # measured DRAM bytes of the analysis kernel scaled to the step's launches (N^2 x maps)
    assert roof["traffic"] == pytest.approx(1027.5e6 * ((2048 / 1024) ** 2 + (8 / 1024) ** 2 + (4 / 1024) ** 2))
    assert set(leg) == {"leg_anal", "leg_synth"}
    assert leg["leg_synth"]["frac"] == pytest.approx(250.0 / tf32)
    assert leg["leg_anal"]["recurrence_tflops"] == pytest.approx(1e13 / 64 / 0.050 / 1e12)
    q = recs["theta_quad"]
    assert q["bound"] == "hbm" and q["unit"] == "GB/s" and q["achieved"] == pytest.approx(400.0)
    assert q["frac"] == pytest.approx(400.0 / 6000.0)
    dense = 4.0 * (2048 ** 3 + 8 ** 3 + 4 ** 3) * 64
    assert q["dense_equivalent_tflops"] == pytest.approx(dense / (15.0 / 1000) / 1e12)
    assert recs["ring_fwd"]["achieved"] == pytest.approx(3000.0) and "pack" not in recs
    # FP32 plans: the Legendre stages against the FP32 pipe, no MMA figure; fallback peaks
    a32 = types.SimpleNamespace(steps=steps, precision="fp32")
    roof32, leg32, _ = bench.rooflines(stats, a32, {}, 64, [2048])
    fp32 = 152 * 128 * 2 * 2070.0 * 1e6 / 1e12
    assert roof32["bound"] == "alu" and roof32["peak"] == pytest.approx(fp32)
    assert "executed_mma_frac" not in roof32 and "of fallback" in roof32["peak_source"]
    # a byte-bound stage that dominates is reported against HBM
    stats2 = dict(stats, ring_fwd=dict(launches=4, timed=4, ms=90.0, flops=0.0, bytes=60e9))
    roof2, _, _ = bench.rooflines(stats2, a, peaks, 64, [2048])
    assert roof2["kernel"] == "ring_fwd" and roof2["bound"] == "hbm" and roof2["traffic"] is None
    assert roof2["frac"] == pytest.approx(60e9 / 0.090 / 1e9 / 6000.0)
    # Legendre stages on the plan's tables: the table bytes they stream per step
    # against HBM; DRAM traffic only from a capture of that kernel variant
    per = {2048: 9e9, 8: 1e6, 4: 0}
    tabs = {"leg_anal": ("table", 30e9, per), "leg_synth": ("table", 30e9, per)}
    roof3, leg3, _ = bench.rooflines(stats, a, peaks, 64, [2048, 8, 4], tabs)
    assert roof3["legendre_values"] == "table"
    # the table kernels contract FP16 hi/lo parts: measured against the FP16 (= BF16) peak
    assert roof3["peak"] == pytest.approx(1800.0) and roof3["frac"] == pytest.approx(200.0 / 1800.0)
    assert roof3["executed_mma_frac"] == pytest.approx(3 * 200.0 / 1800.0) and "FP16" in roof3["peak_source"]
    assert roof3["table_gbs"] == pytest.approx(30e9 / 0.025 / 1e9)
    assert roof3["table_frac_of_hbm"] == pytest.approx(1200.0 / 6000.0)
    # no capture of the table kernels as they are: no traffic
    assert ("leg_anal", "table") not in bench.TRAFFIC and roof3["traffic"] is None
    # with a capture, the traffic of the table kernels is the table copy per launch
    # plus the rest of the captured launch scaled by N^2 x maps
    n0, b0, by = 1024, 64, 2.8e9
    monkeypatch.setitem(bench.TRAFFIC, ("leg_anal", "table"), {"bytes_at": (n0, b0, by), "source": "a capture"})
    per1 = dict(per)
    per1[n0] = 2e9
    roof4, _, _ = bench.rooflines(stats, a, peaks, 64, [2048, 8, 4],
                                  {"leg_anal": ("table", 30e9, per1), "leg_synth": ("table", 30e9, per1)})
    rest = by - 2e9
    want = sum(per1[n] + rest * (n / n0) ** 2 * 64 / b0 for n in (2048, 8, 4))
    assert roof4["traffic"] == pytest.approx(want)
    assert roof3["traffic"] is None
    # two maps sharing a launch read the table once and their data twice
    launches = [(2048, 1), (2048, 2), (8, 1), (4, 1)]
    roof5, _, _ = bench.rooflines(stats, a, peaks, 64, [2048, 2048, 2048, 8, 4],
                                  {"leg_anal": ("table", 30e9, per1, launches),
                                   "leg_synth": ("table", 30e9, per1, launches)})
    want5 = sum(per1[n] + k * rest * (n / n0) ** 2 * 64 / b0 for n, k in launches)
    assert roof5["traffic"] == pytest.approx(want5)
    assert roof5["traffic_gbs"] == pytest.approx(want5 / 0.025 / 1e9)
    assert roof5["traffic_frac_of_hbm"] == pytest.approx(want5 / 0.025 / 1e9 / 6000.0)


def test_legendre_launches_pair_maps_at_one_band_limit():
    """The bench counts the Legendre launches of a round trip as the library runs
    them: the SHT at L, then the maps from scale J down (the scaling map last),
    two neighbours that share a band-limit on the table kernels in one launch."""
    import types
    sys.path.insert(0, ROOT)
    import bench
    L = 2048
    ns = [min(L, 2 ** (j + 1)) for j in range(2, 12)]
    tun = {n: {"table_anal": True, "table_synth": n != 1024} for n in set(ns) | {L, 4}}
    plan = types.SimpleNamespace(L=L, N_scal=4, scales=[(j, n, 0, 0) for j, n in zip(range(2, 12), ns)],
                                 tuning=lambda: tun)
    want = [(L, 1), (L, 2)] + [(n, 1) for n in ns[::-1][2:]] + [(4, 1)]
    assert bench.legendre_launches(plan, "table_synth") == want
    # full resolution: every scale at L, paired two by two, the last one alone
    full = types.SimpleNamespace(L=64, N_scal=64, scales=[(j, 64, 0, 0) for j in range(0, 7)],
                                 tuning=lambda: {64: {"table_anal": True, "table_synth": True}})
    assert bench.legendre_launches(full, "table_anal") == [(64, 1), (64, 2), (64, 2), (64, 2), (64, 2)]
    # no tables at the band-limit: one launch per map
    rec = types.SimpleNamespace(L=64, N_scal=64, scales=[(j, 64, 0, 0) for j in range(0, 3)],
                                tuning=lambda: {64: {"table_anal": False, "table_synth": False}})
    assert bench.legendre_launches(rec, "table_anal") == [(64, 1)] * 5

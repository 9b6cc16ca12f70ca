#!/usr/bin/env python3
"""Benchmark: batched axisymmetric wavelet round trips (analysis then synthesis)
on MW-sampled spheres, one step = one round trip of a batch of real maps at
L = 2048, B = 2, J_min = 2, multiresolution (64 maps per GPU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--L L --B B --J-min J0 --full-res --kernel sd|bspline]   (other workloads)

Prints one JSON line (rank 0).  Inputs are seeded synthetic maps: Gaussian
f_lm with C_l = 1/(l(l+1)), turned into maps by the library's inverse
transform before timing (as the paper's validation does).  The map batch
(2.1 GB in FP32) is far larger than the 129 MB L2, so no flush is needed.
Multi-GPU: each rank transforms its own 64 maps (weak scaling, no collective
on the data path); the elapsed time is the maximum over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "wavelet round-trips/s, L=2048x64 maps, vs plain FP64 GPU path; max err vs oracle"
UNIT = "map round-trips/s"
SM_COUNT = 152
FP32_LANES = 128
FP64_FMA_PER_SM = 2            # FP64 FMA per clock per SM (GB300: 1.25 TFLOP/s FP64 nominal)
TF32_PER_BF16 = 1.1 / 2.25     # nominal dense tensor rates (PFLOP/s per GPU)
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
# what each stage's algorithmic work is (the method's, not the kernels'):
WORK = {
    "ring_fwd": "bytes: the map read and its order-major spectrum F_m(theta_t) written",
    "ring_inv": "bytes: the order-major spectrum read and the map written",
    "theta_quad": "bytes: F_m(theta_t) read and G_m(theta_t) written (an O(N^2 log N) stage)",
    "leg_anal": "flops: 4 per (l, m, ring, map) product of the contraction",
    "leg_synth": "flops: 4 per (l, m, ring, map) product of the contraction",
    "pack": "bytes: none counted (layout conversion of f_lm)",
}
# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# stage's kernel at band-limit N with `batch` maps, from one capture of the kernel
# as it is now, scaled by N^2 x maps (the stage's data grow so); keyed by stage and
# by the Legendre kernel variant in use ("recurrence": the float-float recurrence
# kernels, "table": the kernels that stream the plan's Legendre tables).  A stage
# or variant missing here has no capture of its current kernel, and its traffic
# is reported as null
# The table kernels have no entry: their one capture (profiles/leg_h16_L1024_b64.md)
# predates later changes to them and the two-map kernels were not captured.
TRAFFIC = {
    # k_leg_anal_tc, full-band-limit launch at L = 1024, 64 maps: 772.0 + 255.5 MB
    # (G and the recurrence tables read, f_lm written), profiles/quad_anal_tc_L1024_b64_tf32x3.md
    ("leg_anal", "recurrence"): {
        "bytes_at": (1024, 64, 1027.5e6),
        "source": "ncu dram read+write of k_leg_anal_tc at L=1024 x 64 maps (1027.5 MB per launch), "
                  "scaled by N^2 x maps to every launch of the step"},
}

# noise level of the --denoise steps: white noise of this harmonic standard
# deviation would be thresholded at 3 sigma^j; against the C_l = 1/(l(l+1)) maps
# it zeroes a large part of the fine-scale samples
DENOISE_SIGMA = 1e-3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--precision", choices=["fp32", "tf32x3", "fp64"], default="tf32x3")
    ap.add_argument("--quad-fft64", action="store_true", help="FP32 plans: theta quadrature by FP64 FFTs")
    ap.add_argument("--tc-split3", action="store_true", help="tf32x3 plans: three-part TF32 split (6 MMAs)")
    ap.add_argument("--L", type=int, default=2048)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--B", type=int, default=2)
    ap.add_argument("--J-min", type=int, default=2)
    ap.add_argument("--kernel", choices=["sd", "bspline"], default="sd",
                    help="generating functions: smooth scale-discretised (sd) or cubic B-spline")
    ap.add_argument("--denoise", action="store_true",
                    help="each step denoises (Sect. 4.3): analysis, hard thresholding of the wavelet maps at "
                         "3 sigma^j, synthesis")
    ap.add_argument("--full-res", action="store_true",
                    help="every wavelet and scaling map at L (the full-resolution transform) instead of the "
                         "multiresolution band-limits min(L, B^(j+1))")
    ap.add_argument("--fp64-batch", type=int, default=8)
    ap.add_argument("--fp64-trips", type=int, default=3, help="timed round trips of the plain FP64 GPU path")
    ap.add_argument("--cpu-orders", type=int, default=128)
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="autotune the plan (kernel choice per stage and band-limit) before the warm-up")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-check", action="store_true")
    ap.add_argument("--workload", choices=["l2048x64", "batch256", "grad"], default="l2048x64",
                    help="batch256: 256 complex maps of uneven L in {128..2048} and B in {2, 3}, J_min=1, "
                         "one graph launch per round trip; grad: the loss sum_j 2^-j ||W^j||^2 and its "
                         "gradient (adjoint kernel) at L=1024 x 16 real maps, and with per-scale "
                         "recomputation for one map at L=4096")
    return ap.parse_args()


def config(a):
    return {"workload": "real maps, L=%d, B=%d, J_min=%d, %s%s, %d maps per GPU, f_lm ~ C_l=1/(l(l+1))"
                        % (a.L, a.B, a.J_min, "full resolution" if a.full_res else "multiresolution",
                           ", B-spline kernels" if a.kernel == "bspline" else "", a.batch),
            "kernel": a.kernel, "denoise": a.denoise,
            "L": a.L, "B": a.B, "J_min": a.J_min, "maps_per_gpu": a.batch, "multires": not a.full_res,
            "signal": "real",
            "precision": a.precision + ("+quad_fft64" if a.quad_fft64 else "") + ("+split3" if a.tc_split3 else ""),
            "l2": "inputs larger than L2 (map batch %.2f GB)" % (a.batch * a.L * (2 * a.L - 1)
                                                                   * (8 if a.precision == "fp64" else 4) / 1e9)}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- oracle legs
def oracle_sample_step(f, a, orders):
    """One step of the CPU oracle: analysis then synthesis of one map at the
    full workload size, restricted to the given orders m (both transforms act
    on each order separately)."""
    import oracle.wavelet as ow
    fw, fs = ow.analysis(f, a.L, a.B, a.J_min, not a.full_res, False, orders=orders, kernel=a.kernel)
    ow.synthesis(fw, fs, a.L, a.B, a.J_min, not a.full_res, False, orders=orders, kernel=a.kernel)


def oracle_input(a, seed):
    import oracle.sht as osht
    from paper_1211_1680_gb300 import inputs
    return osht.inverse(inputs.random_flm(a.L, seed, True, "cl"), a.L, real=True)


def cpu_baseline(a, steps=1, warmup=1):
    """Oracle timed on this host's cores on a bounded sample of the workload."""
    import oracle.sht as osht
    rng = np.random.default_rng(12345)
    f = np.random.default_rng(7).standard_normal((a.L, 2 * a.L - 1))   # values do not change the cost
    for N in sorted({a.L} | {min(a.L, a.B ** (j + 1)) for j in range(a.J_min, 20)} | {min(a.L, a.B ** a.J_min)}):
        osht._quadrature_matrices(N)
        osht._phase_matrix_phi(N)
    all_orders = np.arange(-(a.L - 1), a.L)
    for _ in range(warmup):
        oracle_sample_step(f, a, rng.choice(all_orders, size=min(a.cpu_orders, len(all_orders)), replace=False))
    t = 0.0
    for _ in range(steps):
        orders = rng.choice(all_orders, size=min(a.cpu_orders, len(all_orders)), replace=False)
        t0 = time.perf_counter()
        oracle_sample_step(f, a, orders)
        t += time.perf_counter() - t0
    frac = steps * len(orders) / len(all_orders)
    value = frac / t
    return {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle analysis+synthesis of 1 map at L=%d restricted to %d random orders m of %d "
                      "(every stage acts on each order separately); value = (orders/%d) / time; %d step(s); "
                      "matrix products on %d rows run below their all-rows efficiency, so this understates "
                      "the oracle" % (a.L, len(orders), len(all_orders), len(all_orders), steps, len(orders)),
            "seconds": t}


def run_reference(a, rank):
    if rank != 0:
        return 0
    import oracle.sht as osht
    rng = np.random.default_rng(4242)
    f = np.random.default_rng(7).standard_normal((a.L, 2 * a.L - 1))
    for N in sorted({a.L} | {min(a.L, a.B ** (j + 1)) for j in range(a.J_min, 20)} | {min(a.L, a.B ** a.J_min)}):
        osht._quadrature_matrices(N)
        osht._phase_matrix_phi(N)
    all_orders = np.arange(-(a.L - 1), a.L)
    k = min(a.cpu_orders, len(all_orders))
    for _ in range(a.warmup):
        oracle_sample_step(f, a, rng.choice(all_orders, size=k, replace=False))
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle_sample_step(f, a, rng.choice(all_orders, size=k, replace=False))
    t = time.perf_counter() - t0
    value = a.steps * k / len(all_orders) / t
    sample = ("each step: oracle analysis+synthesis of 1 map at L=%d restricted to %d random orders of %d; "
              "value = (orders/%d) / time" % (a.L, k, len(all_orders), len(all_orders)))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * t / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(a),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- rooflines
def peak_table(peaks):
    """Peaks used for the roofline fractions: the measured ones where
    MEASURED_PEAKS.json holds them, else the fallback figures; each with its source."""
    def get(k):
        if k in peaks:
            return float(peaks[k]), "of measured"
        return FALLBACK[k], "of fallback"
    hbm, hsrc = get("hbm_gbs")
    bf, bsrc = get("bf16_tflops_sustained")
    mhz, msrc = get("sm_max_mhz")
    return {
        "hbm": (hbm, "GB/s", "HBM copy bandwidth hbm_gbs %.0f GB/s (%s)" % (hbm, hsrc)),
        "tf32": (bf * TF32_PER_BF16, "TFLOP/s",
                 "TF32 dense = bf16_tflops_sustained %.1f (%s) x 1.1/2.25 (nominal TF32/BF16 ratio)" % (bf, bsrc)),
        "f16": (bf, "TFLOP/s",
                "FP16 dense = bf16_tflops_sustained %.1f (%s) (FP16 and BF16 share one nominal rate)" % (bf, bsrc)),
        "fp32": (SM_COUNT * FP32_LANES * 2 * mhz * 1e6 / 1e12, "TFLOP/s",
                 "derived: %d SMs x %d FP32 lanes x 2 flop/FMA x %.0f MHz (%s)" % (SM_COUNT, FP32_LANES, mhz, msrc)),
        "fp64": (SM_COUNT * FP64_FMA_PER_SM * 2 * mhz * 1e6 / 1e12, "TFLOP/s",
                 "derived: %d SMs x %d FP64 FMA/clk x 2 flop x %.0f MHz (%s)" % (SM_COUNT, FP64_FMA_PER_SM, mhz, msrc)),
    }


def legendre_launches(plan, key):
    """The Legendre launches of one round trip in one direction, as (band-limit,
    maps per launch): the SHT at L, and one per wavelet or scaling map, where
    two maps next to each other in the library's processing order (scale J
    first, the scaling map last) that share a band-limit on the table kernels
    share one launch (one table stream for both)."""
    tun = plan.tuning()
    order = [n for (_, n, _, _) in sorted(plan.scales, reverse=True)] + [plan.N_scal]
    out = [(plan.L, 1)]
    i = 0
    while i < len(order):
        n = order[i]
        if i + 1 < len(order) and order[i + 1] == n and tun[n][key]:
            out.append((n, 2))
            i += 2
        else:
            out.append((n, 1))
            i += 1
    return out


def legendre_tables(plan):
    """Per Legendre stage: which values it contracts ("table": the plan's stored
    Legendre tables, "recurrence": computed in the kernel) at the full band-limit,
    the table bytes its launches of one round trip read, the bytes one launch
    reads at each band-limit (one of the two copies the plan stores: rows =
    degrees for the analysis, rows = rings for the synthesis; 0 where the stage
    runs the recurrence), and its launches as (band-limit, maps per launch)."""
    if plan.precision != "tf32x3":
        return {}
    tun = plan.tuning()
    out = {}
    for stage, key in (("leg_anal", "table_anal"), ("leg_synth", "table_synth")):
        variant = "table" if tun[plan.L][key] else "recurrence"
        per = {n: (plan.table_bytes(n) // 2 if tun[n][key] else 0) for n in set(plan_bandlimits(plan))}
        launches = legendre_launches(plan, key)
        out[stage] = (variant, sum(per[n] for n, _ in launches), per, launches)
    return out


def dtype_of(precision, plan=None):
    """Arithmetic types of the path: split tensor-core plans contract in FP16 hi/lo
    where they stream Legendre tables, in split TF32 elsewhere (the recurrence
    kernels, the dense quadrature), with FP32 FFTs.  Without a plan to ask (the
    batch and gradient workloads), the types of a default plan, which stores the
    tables of band-limits up to 2048."""
    if precision == "tf32x3":
        if plan is None or any(t["table_anal"] or t["table_synth"] for t in plan.tuning().values()):
            return "f16x3+tf32x3+f32"
        return "tf32x3+f32"
    return {"fp32": "f32", "fp64": "f64"}[precision]


def plan_bandlimits(plan):
    """Band-limits of the transforms in one round trip: each direction runs one
    SHT at L and one per wavelet or scaling map."""
    return [plan.L] + [n for (_, n, _, _) in plan.scales] + [plan.N_scal]


def stage_roofline(name, st, steps, precision, pk, batch, variant="recurrence"):
    """Roofline record of one stage from its per-stage statistics: achieved =
    algorithmic work / device time (all launches of the stage, so the average
    over its launches weighted by their duration).  variant: the Legendre values
    of a split tensor-core plan's stage ("table": the FP16 hi/lo kernels on the
    plan's tables, measured against the FP16 peak; "recurrence": the split-TF32
    kernels, against the TF32 peak)."""
    sec = st["ms"] / 1000.0
    if sec <= 0:
        return None
    rec = {"ms_per_step": st["ms"] / steps, "launches_per_step": st["launches"] / steps, "work": WORK.get(name, "")}
    if st["flops"] > 0:
        key = {"tf32x3": "tf32", "fp32": "fp32", "fp64": "fp64"}[precision]
        if key == "tf32" and variant == "table":
            key = "f16"
        peak, unit, src = pk[key]
        achieved = st["flops"] / sec / 1e12
        tensor = key in ("tf32", "f16")
        rec.update(bound="tensor" if tensor else "alu", achieved=achieved, peak=peak, unit=unit,
                   frac=achieved / peak, peak_source=src)
        if tensor:
            rec["executed_mma_frac"] = 3.0 * achieved / peak
            rec["executed_note"] = ("split %s runs 3 MMAs per algorithmic product (hi*hi + hi*lo + lo*hi)"
                                    % ("FP16" if key == "f16" else "TF32"))
        # the three-term recurrence behind the products: 4 flops per lambda value; real
        # maps share one value among the batch's maps (and re/im), so per step it is
        # the contraction's count divided by the maps
        rflops = st["flops"] / batch
        rec["recurrence_tflops"] = rflops / sec / 1e12
        rec["recurrence_frac_of_fp32_pipe"] = rflops / sec / 1e12 / pk["fp32"][0]
    else:
        peak, unit, src = pk["hbm"]
        achieved = st["bytes"] / sec / 1e9
        rec.update(bound="hbm", achieved=achieved, peak=peak, unit=unit, frac=achieved / peak, peak_source=src)
    return rec


def rooflines(stats, a, peaks, batch, bandlimits, tables=None):
    """(roofline of the dominant stage, Legendre sub-record, every stage's record).
    tables: {stage: (variant, table bytes read per step)} of the Legendre stages."""
    pk = peak_table(peaks)
    tables = tables or {}
    recs = {k: stage_roofline(k, v, a.steps, a.precision, pk, batch, tables.get(k, ("recurrence", 0))[0])
            for k, v in stats.items() if v["launches"]}
    tables = {k: (t + ({}, None))[:4] for k, t in tables.items()}
    recs = {k: v for k, v in recs.items() if v is not None}
    for k, (variant, tbytes, _, _) in tables.items():
        if k in recs:
            recs[k]["legendre_values"] = variant
            if tbytes:
                # the tables are streamed from HBM once per launch
                recs[k]["table_bytes_per_step"] = tbytes
                recs[k]["table_gbs"] = tbytes / (recs[k]["ms_per_step"] / 1000) / 1e9
                recs[k]["table_frac_of_hbm"] = recs[k]["table_gbs"] / pk["hbm"][0]
    dom = max(recs, key=lambda k: recs[k]["ms_per_step"])
    roof = dict(recs[dom])
    roof["kernel"] = dom
    variant, _, per, launches = tables.get(dom, ("recurrence", 0, {}, None))
    tr = TRAFFIC.get((dom, variant)) if a.precision == "tf32x3" else None
    if tr and variant == "table" and tr["bytes_at"][0] in per:
        # table kernels: the table part of a launch is the copy it streams (grows as
        # the table, ~N^3), once per launch even where two maps share it; the rest
        # (data read, results written) as N^2 x maps, per map of the launch
        n0, b0, by = tr["bytes_at"]
        rest = by - per[n0]
        launches = launches or [(n, 1) for n in bandlimits]
        roof["traffic"] = sum(per.get(n, 0) + sets * rest * (n / n0) ** 2 * batch / b0 for n, sets in launches)
        roof["traffic_note"] = tr["source"]
    elif tr and variant != "table":
        n0, b0, by = tr["bytes_at"]
        # one launch of the stage per transform direction and band-limit of the round trip
        roof["traffic"] = sum(by * (n / n0) ** 2 * batch / b0 for n in bandlimits)
        roof["traffic_note"] = tr["source"]
        roof["traffic_vs_algorithmic_note"] = ("the Legendre stages have no algorithmic bytes of their own "
                                               "(contraction flops are their work); traffic is the G and table "
                                               "reads and f_lm writes")
    else:
        roof["traffic"] = None
    if roof["traffic"] and variant == "table":
        # the table kernels are bound by HBM (64 flop per table byte, 128 where two maps
        # share a stream, below the FP16 ridge): their DRAM traffic against the HBM peak
        sec = roof["ms_per_step"] / 1000.0
        roof["traffic_gbs"] = roof["traffic"] / sec / 1e9
        roof["traffic_frac_of_hbm"] = roof["traffic_gbs"] / pk["hbm"][0]
    roof["note"] = "achieved and traffic are per step of the stage (all its launches)"
    # the dense theta-quadrature products of FP32 / TF32X3 plans, as a labelled extra
    if "theta_quad" in recs and a.precision != "fp64":
        dense = sum(4.0 * n ** 3 * batch for n in bandlimits)   # forward SHTs: 2 N^2 per real column
        recs["theta_quad"]["dense_equivalent_tflops"] = dense / (recs["theta_quad"]["ms_per_step"] / 1000) / 1e12
        recs["theta_quad"]["dense_equivalent_note"] = ("if the stage ran as the dense product G = Q F at every "
                                                       "band-limit: 2 N^2 flops per real column")
    legendre = {k: recs[k] for k in ("leg_anal", "leg_synth") if k in recs}
    return roof, legendre, recs


# ---------------------------------------------------------------- GPU leg
def check_errors(plan, x, fw, fs, out, flm, a):
    """Per-scale max relative error of map 0 against the oracle, on sampled rings:
    W^j(theta_t, phi_p) = sum_lm kappa(l/B^j) f_lm Y_lm (Eq. wav2) from the
    input coefficients; plus the round-trip reconstruction error."""
    import oracle.sht as osht
    import oracle.wavelet as ow
    phi, psi = ow.tables(a.L, a.B, a.J_min, a.kernel)
    res = {}
    views = plan.wavelet_views(fw)
    maps = [("scal", plan.N_scal, phi, fs)] + [("j%d" % j, n, p, v) for (j, n, _, _), p, v in
                                               zip(plan.scales, psi, views)]
    l_of = np.repeat(np.arange(a.L), 2 * np.arange(a.L) + 1)
    norm = np.sqrt(4 * np.pi / (2 * l_of + 1))
    xmax = x[0].detach().double().abs().max().item()
    for name, n, kern, v in maps:
        wlm = (norm * flm * kern[l_of])[:n * n]
        rings = sorted({0, 1, n // 3, n // 2, n - 2, n - 1} & set(range(n)))
        ref = osht.inverse_at(wlm, n, rings, np.arange(2 * n - 1)).real
        got = v[0].detach().double().cpu().numpy()[rings]
        # a scale whose band holds no power of the input (C_0 = C_1 = 0 leaves the
        # scaling map and scale 0 of J_min = 0 exactly zero) has no scale of its own:
        # its rounding residue is measured against the input map instead
        full = v[0].detach().double().abs().max().item() if np.any(wlm) else xmax
        res[name] = float(np.max(np.abs(got - ref)) / max(full, 1e-300))
    rec = float(((out[0] - x[0]).abs().max() / x[0].abs().max()).item())
    return {"max_rel_err_by_scale": res, "max_rel_err": max(res.values()), "round_trip_rel_err": rec,
            "check": "map 0; rings {0,1,N/3,N/2,N-2,N-1} of every scale against the oracle's direct sum; "
                     "error normalised by the scale map's max (by the input map's max for a scale whose "
                     "band holds no input power)"}


def run_gpu(a, rank, world, local_rank):
    import torch
    from paper_1211_1680_gb300 import inputs
    from paper_1211_1680_gb300.s2let import Plan

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    seeds = [3000 + rank * a.batch + i for i in range(a.batch)]
    flm = inputs.random_flm_batch(a.L, seeds, real=True, kind="cl")
    plan = Plan(a.L, a.B, a.J_min, batch=a.batch, real=True, multires=not a.full_res, precision=a.precision,
                kernel=a.kernel,
                quad_fft64=a.quad_fft64, tc_split3=a.tc_split3)
    flm_d = torch.from_numpy(np.stack([flm.real, flm.imag], -1)).to(device="cuda", dtype=plan.dtype).contiguous()
    x = plan.sht_inverse(flm_d)
    del flm_d
    fw, fs = plan.empty_wavelets()
    out = plan.empty_map()
    stream = torch.cuda.current_stream()
    tuning = plan.autotune() if a.autotune else None

    def step(src=x, dst=out):
        plan.analysis(src, fw, fs)
        if a.denoise:
            plan.threshold(fw, DENOISE_SIGMA)
        plan.synthesis(fw, fs, dst)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    plan.profile(True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stats = plan.stage_stats()
    plan.profile(False)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        ms = float(t.item())
    value = world * a.batch * a.steps / (ms / 1000.0)

    roof, legendre, all_stages = rooflines(stats, a, measured_peaks(), a.batch, plan_bandlimits(plan),
                                           legendre_tables(plan))
    total_ms = sum(s["ms"] for s in stats.values())
    stage_share = {k: {"share": (s["ms"] / total_ms if total_ms else 0.0), "ms_per_step": s["ms"] / a.steps,
                       "launches_per_step": s["launches"] / a.steps} for k, s in stats.items()}
    launches = sum(s["launches"] for s in stats.values())

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype_of(a.precision, plan), "data": "synthetic",
           "config": config(a),
           "gpu_launches": launches, "roofline": roof, "legendre": legendre, "stage_rooflines": all_stages,
           "stages": stage_share, "clocks": clk}
    if tuning is not None:
        res["tuning"] = {str(n): t for n, t in tuning.items()}

    # end to end: pinned host maps in, host maps out, copies inside the timed region.
    # Every step copies its input batch in and its result batch out; the copies of
    # neighbouring steps run on two copy streams while a step computes
    # (s2let.HostPipeline), so only the first copy-in and the last copy-out are exposed.
    if not a.skip_e2e:
        from paper_1211_1680_gb300.s2let import HostPipeline
        xh = x.cpu().pin_memory()
        oh = [torch.empty_like(out, device="cpu").pin_memory() for _ in range(2)]
        pipe = HostPipeline(x, out)

        def e2e(n):
            pipe.run(n, lambda k: xh, lambda k: oh[k % 2], lambda src, dst: step(src, dst))

        e2e(2)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e(a.e2e_steps)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        if dist:
            t = torch.tensor([te], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        # the copies alone, for the record (same pinned buffers, one of each direction)
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record(stream)
        pipe.din[0].copy_(xh, non_blocking=True)
        c1.record(stream)
        oh[0].copy_(pipe.dout[0], non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize()
        res["e2e"] = {"value": world * a.batch * a.e2e_steps / te, "unit": UNIT,
                      "h2d_bytes_per_step": xh.numel() * xh.element_size(),
                      "d2h_bytes_per_step": oh[0].numel() * oh[0].element_size(),
                      "steps": a.e2e_steps, "overlap": "copy-in of step k+1 and copy-out of step k-1 on two copy "
                                                       "streams while step k computes",
                      "h2d_gbs_alone": xh.numel() * xh.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9,
                      "d2h_gbs_alone": xh.numel() * xh.element_size() / (c1.elapsed_time(c2) / 1e3) / 1e9}
        del pipe

    if rank == 0 and not a.skip_check:
        if a.denoise:
            # the check compares the transform itself: one round trip without thresholding
            plan.analysis(x, fw, fs)
            plan.synthesis(fw, fs, out)
            torch.cuda.synchronize()
        res.update(check_errors(plan, x, fw, fs, out, flm[0], a))

    # the plain FP64 GPU path on the same workload (fewer maps per launch)
    if rank == 0 and not a.skip_fp64 and a.precision != "fp64":
        del fw, fs, out
        nb = a.fp64_batch
        p64 = Plan(a.L, a.B, a.J_min, batch=nb, real=True, multires=not a.full_res, precision="fp64",
                   kernel=a.kernel)
        f64 = torch.from_numpy(np.stack([flm[:nb].real, flm[:nb].imag], -1)).cuda().contiguous()
        x64 = p64.sht_inverse(f64)
        w64, s64 = p64.empty_wavelets()
        o64 = p64.empty_map()
        p64.analysis(x64, w64, s64)
        p64.synthesis(w64, s64, o64)
        torch.cuda.synchronize()
        trips = []
        for _ in range(a.fp64_trips):
            e0.record(stream)
            p64.analysis(x64, w64, s64)
            p64.synthesis(w64, s64, o64)
            e1.record(stream)
            torch.cuda.synchronize()
            trips.append(e0.elapsed_time(e1) / 1000.0)
        t64 = statistics.median(trips)
        v64 = nb / t64
        res["fp64_path"] = {"value": v64, "unit": UNIT, "maps": nb, "ms_per_round_trip": 1000 * t64,
                            "ms_per_round_trip_each": [1000 * t for t in trips],
                            "spread": (max(trips) - min(trips)) / t64,
                            "note": "plain FP64 GPU path, same L/B/J_min, %d maps per launch; median of %d timed "
                                    "round trips after one warm-up" % (nb, len(trips))}
        res["speedup_vs_fp64_path"] = value / world / v64
        del p64

    if rank == 0 and not a.skip_cpu:
        res["cpu_baseline"] = cpu_baseline(a)
    if rank == 0:
        print(json.dumps(res), flush=True)
    return 0


def run_batch256(a, rank, world, local_rank):
    """256 complex maps, L ~ {128: .3, 256: .3, 512: .2, 1024: .1, 2048: .1}, B ~ {2, 3}, J_min = 1,
    FP32; every round trip of the whole uneven batch is one CUDA graph launch."""
    import ctypes
    import torch
    from paper_1211_1680_gb300 import _lib, inputs
    from paper_1211_1680_gb300.s2let import BatchPlan

    torch.cuda.set_device(local_rank)
    rng = np.random.Generator(np.random.PCG64(4 + rank))
    Ls = rng.choice([128, 256, 512, 1024, 2048], size=256, p=[0.3, 0.3, 0.2, 0.1, 0.1]).tolist()
    Bs = rng.choice([2, 3], size=256).tolist()
    prec = a.precision
    bp = BatchPlan(Ls, Bs, 1, real=False, multires=True, precision=prec)
    f, fw, fs, fo = bp.buffers()
    lib = _lib.lib()
    # inputs: per group, seeded complex Gaussian f_lm -> maps with the group plan's inverse transform
    kept = {}                          # the first map of each group: its coefficients, for the oracle check
    for g, (ph, f_off, _, _) in enumerate(bp.groups):
        members = [i for i in range(256) if bp.layout[i][2] == g]
        L = Ls[members[0]]
        flm = np.stack([inputs.random_flm(L, 4000 + rank * 256 + i, real=False) for i in members])
        kept[members[0]] = flm[0]
        fl = torch.from_numpy(np.stack([flm.real, flm.imag], -1)).to("cuda", bp.dtype).contiguous()
        n = len(members) * L * (2 * L - 1) * 2
        check = lib.s2let_sht_inverse(ctypes.c_void_p(ph), ctypes.c_void_p(fl.data_ptr()),
                                      ctypes.c_void_p(f[f_off:f_off + n].data_ptr()), None)
        assert check == 0
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            bp.round_trip(f, fw, fs, fo)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(local_rank)
        clocks.start()
        e0.record(stream)
        for _ in range(a.steps):
            bp.round_trip(f, fw, fs, fo)
        e1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    err = max(float(((bp.map_view(fo, i) - bp.map_view(f, i)).abs().max() / bp.map_view(f, i).abs().max()).item())
              for i in range(256))
    hist = {int(L): Ls.count(L) for L in sorted(set(Ls))}
    # the wavelet maps of the first map of every group against the oracle's direct sum
    # of Eq. wav2 on sampled rings (every scale), as in the main workload's check
    wav_err = 0.0
    if rank == 0 and not a.skip_check:
        import oracle.sht as osht
        import oracle.wavelet as ow
        for i, flm in kept.items():
            L, B = Ls[i], Bs[i]
            _, _, g, k = bp.layout[i]
            ph, _, wav_off, _ = bp.groups[g]
            _, psi = ow.tables(L, B, 1)
            l_of = np.repeat(np.arange(L), 2 * np.arange(L) + 1)
            norm = np.sqrt(4 * np.pi / (2 * l_of + 1))
            for j, kern in zip(range(1, 1 + len(psi)), psi):
                n_, off_, cnt_ = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
                assert lib.s2let_wav_layout(ctypes.c_void_p(ph), j, ctypes.byref(n_), ctypes.byref(off_),
                                            ctypes.byref(cnt_)) == 0
                n = n_.value
                per = n * (2 * n - 1) * 2
                start = wav_off + off_.value + k * per
                v = fw[start:start + per].view(n, 2 * n - 1, 2).double().cpu().numpy()
                v = v[..., 0] + 1j * v[..., 1]
                rings = sorted({0, 1, n // 3, n // 2, n - 2, n - 1} & set(range(n)))
                ref = osht.inverse_at((norm * flm * kern[l_of])[:n * n], n, rings, np.arange(2 * n - 1))
                wav_err = max(wav_err, float(np.max(np.abs(v[rings] - ref)) / np.max(np.abs(v))))
    res = {"metric": "uneven-batch wavelet round-trips/s (256 complex maps, one graph launch per round trip)",
           "value": world * 256 * a.steps / (ms / 1000.0), "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dtype_of(prec),
           "data": "synthetic",
           "config": {"workload": "256 complex maps, L histogram %s, B in {2,3}, J_min=1, multiresolution" % hist,
                      "groups": bp.n_groups, "graph_launches_per_step": 1},
           "round_trip_rel_err": err, "clocks": clk,
           "max_rel_err": wav_err,
           "check": "round trip of all 256 maps; wavelet maps (every scale, rings {0,1,N/3,N/2,N-2,N-1}) of "
                    "the first map of each (L, B) group against the oracle's direct sum, normalised by the "
                    "scale map's max"}
    if rank == 0:
        print(json.dumps(res), flush=True)
    return 0


def run_grad(a, rank, world, local_rank):
    """Differentiation workload: loss = sum_j 2^-j ||W^j||^2 (wavelet scales) of real
    maps and its gradient with respect to the maps.  (1) 16 maps at L = 1024, B = 2,
    J_min = 2: backward through the adjoint kernel (s2let_adjoint), and with per-scale
    recomputation; (2) one map at L = 4096 with per-scale recomputation.  A step is
    one forward + backward; the value is maps per second of the first case."""
    import torch
    from paper_1211_1680_gb300 import inputs
    from paper_1211_1680_gb300.autograd import scale_energy_loss, scale_energy_loss_recompute
    from paper_1211_1680_gb300.s2let import Plan

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {}
    for (L, nb, label) in ((1024, 16, "L1024x16"), (4096, 1, "L4096x1")):
        plan = Plan(L, 2, 2, batch=nb, real=True, multires=True, precision=a.precision)
        flm = inputs.random_flm_batch(L, [5000 + rank * nb + i for i in range(nb)], real=True, kind="cl")
        x = plan.sht_inverse(torch.from_numpy(np.stack([flm.real, flm.imag], -1)).to("cuda", plan.dtype)
                             .contiguous())
        f = x.clone().requires_grad_(True)
        rec = {}
        variants = [("recompute", scale_energy_loss_recompute)]
        if L <= 2048:
            variants.insert(0, ("adjoint", scale_energy_loss))
        for name, loss_fn in variants:
            def step():
                loss = loss_fn(f, plan)
                (g,) = torch.autograd.grad(loss, f)
                return g
            torch.cuda.reset_peak_memory_stats()
            ms = timed(step, a.steps, a.warmup)
            rec[name] = {"ms_per_step": ms, "maps_per_s": nb / (ms / 1000.0),
                         "peak_torch_bytes": torch.cuda.max_memory_allocated()}
        if "adjoint" in rec:
            g1 = torch.autograd.grad(scale_energy_loss(f, plan), f)[0]
            g2 = torch.autograd.grad(scale_energy_loss_recompute(f, plan), f)[0]
            rec["recompute_vs_adjoint_rel_diff"] = float(((g2 - g1).abs().max() / g1.abs().max()).item())
        out[label] = rec
        del plan, x, f
        torch.cuda.empty_cache()
    first = out["L1024x16"]["adjoint"]
    res = {"metric": "loss + gradient evaluations of sum_j 2^-j ||W^j||^2 (maps/s), L=1024 x 16 real maps",
           "value": world * first["maps_per_s"], "unit": "maps/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": first["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dtype_of(a.precision),
           "data": "synthetic",
           "config": {"workload": "loss + gradient: L=1024 x 16 real maps (adjoint kernel and per-scale "
                                  "recomputation), L=4096 x 1 map (per-scale recomputation); B=2, J_min=2, "
                                  "f_lm ~ C_l=1/(l(l+1))"},
           "cases": out}
    if rank == 0:
        print(json.dumps(res), flush=True)
    return 0


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    try:
        if a.workload == "batch256":
            return run_batch256(a, rank, world, local_rank)
        if a.workload == "grad":
            return run_grad(a, rank, world, local_rank)
        return run_gpu(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

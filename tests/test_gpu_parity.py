"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Tolerances (max relative error, normwise per result):
1e-10 for FP64 plans, 1e-5 for FP32 and TF32X3 plans."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kernels, sht, wavelet  # noqa: E402
from paper_1211_1680_gb300 import inputs  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402
from tests.gpu_util import TOL, flm_from_dev, flm_to_dev, from_dev_map, plan_kwargs, rel_err, to_dev_map  # noqa: E402


def _maps(L, seeds, real, kind="white"):
    return np.stack([sht.inverse(inputs.random_flm(L, s, real, kind), L, real=real) for s in seeds])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32x3s3", "tf32x3rec"])
@pytest.mark.parametrize("real", [True, False])
@pytest.mark.parametrize("L", [3, 4, 8, 17, 33, 64, 130])
def test_sht_forward_inverse(L, real, prec):
    seeds = [11, 12, 13]
    plan = Plan(L, 2, 0, batch=len(seeds), real=real, multires=True, **plan_kwargs(prec))
    flm = np.stack([inputs.random_flm(L, s, real) for s in seeds])
    f_ref = np.stack([sht.inverse(x, L, real=real) for x in flm])
    # inverse
    f_gpu = from_dev_map(plan.sht_inverse(flm_to_dev(flm, plan.dtype)), real)
    assert rel_err(f_gpu, f_ref) < TOL[prec]
    # forward of the oracle's maps
    g = flm_from_dev(plan.sht_forward(to_dev_map(f_ref, plan.dtype, real)))
    ref = np.stack([sht.forward(x, L) for x in f_ref])
    assert rel_err(g, ref) < TOL[prec]
    assert plan.status() == 0


@pytest.mark.parametrize("real,nb", [(True, 70), (False, 35)])
def test_sht_tensor_core_tiles(real, nb):
    """TF32X3 plan at L = 300 with two batch tiles of the tensor-core Legendre
    kernels: three ring tiles and three degree tiles (ragged), ten ring chunks.
    Slot b holds c_b times one of two oracle transforms."""
    L = 300
    flm = [inputs.random_flm(L, 41 + i, real) for i in range(2)]
    f_ref = [sht.inverse(x, L, real=real) for x in flm]
    c = [(-1.0) ** b * (1.0 + b / nb) for b in range(nb)]
    plan = Plan(L, 2, 0, batch=nb, real=real, precision="tf32x3")
    f_gpu = from_dev_map(plan.sht_inverse(flm_to_dev(np.stack([c[b] * flm[b % 2] for b in range(nb)]), plan.dtype)),
                         real)
    assert rel_err(f_gpu, np.stack([c[b] * f_ref[b % 2] for b in range(nb)])) < TOL["tf32x3"]
    fwd = [sht.forward(x, L) for x in f_ref]
    x = to_dev_map(np.stack([c[b] * f_ref[b % 2] for b in range(nb)]), plan.dtype, real)
    g = flm_from_dev(plan.sht_forward(x))
    assert rel_err(g, np.stack([c[b] * fwd[b % 2] for b in range(nb)])) < TOL["tf32x3"]
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_sht_forward_not_bandlimited(prec):
    """Any samples (pole ring not constant, no band-limit): same linear map."""
    L = 24
    x = np.stack([inputs.random_map((L, 2 * L - 1), s) for s in (5, 6)])
    plan = Plan(L, 2, 0, batch=2, real=True, precision=prec)
    g = flm_from_dev(plan.sht_forward(to_dev_map(x, plan.dtype, True)))
    ref = np.stack([sht.forward(v, L) for v in x])
    assert rel_err(g, ref) < TOL[prec]


CASES = [  # L, B, J0, multires, real, prec
    (32, 2, 0, False, True, "fp64"),      # full-resolution L=32 workload
    (32, 2, 0, True, True, "fp64"),       # scaling map at band-limit 1
    (32, 2, 0, False, True, "fp32"),
    (40, 3, 1, True, False, "fp64"),
    (27, 3, 2, False, False, "fp32"),
    (65, 2, 5, True, True, "fp32"),       # J0 = J - 1
    (3, 2, 0, True, True, "fp64"),        # smallest L
    (96, 2, 2, True, True, "fp64"),
    (96, 2, 2, True, True, "tf32x3"),
    (40, 3, 1, True, False, "tf32x3"),
    (96, 2, 2, True, True, "tf32x3s3"),
    (96, 2, 2, True, True, "tf32x3rec"),
    (40, 3, 1, True, False, "tf32x3rec"),
]


@pytest.mark.parametrize("L,B,J0,multires,real,prec", CASES)
def test_wavelet_analysis_synthesis(L, B, J0, multires, real, prec):
    seeds = [21, 22]
    f = _maps(L, seeds, real)
    plan = Plan(L, B, J0, batch=len(seeds), real=real, multires=multires, **plan_kwargs(prec))
    fw_d, fs_d = plan.analysis(to_dev_map(f, plan.dtype, real))
    ref = [wavelet.analysis(x, L, B, J0, multires, real) for x in f]
    for i, view in enumerate(plan.wavelet_views(fw_d)):
        got = from_dev_map(view, real)
        want = np.stack([r[0][i] for r in ref])
        assert rel_err(got, want) < TOL[prec], "scale %d" % (J0 + i)
    got = from_dev_map(fs_d, real)
    assert rel_err(got, np.stack([r[1] for r in ref])) < TOL[prec]
    # synthesis of the oracle's wavelet maps
    fw_in = torch.cat([to_dev_map(np.stack([r[0][i] for r in ref]), plan.dtype, real).reshape(-1)
                       for i in range(len(ref[0][0]))])
    fs_in = to_dev_map(np.stack([r[1] for r in ref]), plan.dtype, real)
    rec = from_dev_map(plan.synthesis(fw_in, fs_in), real)
    want = np.stack([wavelet.synthesis(r[0], r[1], L, B, J0, multires, real) for r in ref])
    assert rel_err(rec, want) < TOL[prec]
    assert rel_err(rec, f) < TOL[prec]
    assert plan.status() == 0


@pytest.mark.parametrize("L,B,J0,multires,real,prec", [
    (16, 2, 1, True, True, "fp64"), (16, 2, 0, False, False, "fp64"),
    (24, 3, 1, True, True, "fp32"), (33, 2, 2, True, False, "fp32"),
    (24, 3, 1, True, True, "tf32x3"), (140, 2, 2, True, False, "tf32x3"),
])
def test_adjoint_against_oracle(L, B, J0, multires, real, prec):
    plan = Plan(L, B, J0, batch=2, real=real, multires=multires, precision=prec)
    n_scal, n_wav = kernels.bandlimits(L, B, J0, multires)
    gws = [[inputs.random_map((n, 2 * n - 1), 100 * b + i, real) for i, n in enumerate(n_wav)] for b in range(2)]
    gss = [inputs.random_map((n_scal, 2 * n_scal - 1), 77 + b, real) for b in range(2)]
    fw = torch.cat([to_dev_map(np.stack([gw[i] for gw in gws]), plan.dtype, real).reshape(-1)
                    for i in range(len(n_wav))])
    fs = to_dev_map(np.stack(gss), plan.dtype, real)
    got = from_dev_map(plan.adjoint(fw, fs), real)
    want = np.stack([wavelet.analysis_adjoint(gws[b], gss[b], L, B, J0, multires, real) for b in range(2)])
    assert rel_err(got, want) < TOL[prec]
    assert plan.status() == 0


BSPLINE_CASES = [  # L, B, J0, multires, real, prec
    (64, 2, 1, True, True, "fp64"),
    (40, 3, 1, True, False, "fp64"),
    (33, 2, 0, False, True, "fp32"),       # full resolution, odd band-limit
    (96, 2, 2, True, True, "tf32x3"),
    (130, 3, 1, True, False, "tf32x3"),    # band-limits ceil(L / 3^e), not powers of B
]


@pytest.mark.parametrize("L,B,J0,multires,real,prec", BSPLINE_CASES)
def test_bspline_wavelets(L, B, J0, multires, real, prec):
    """B-spline generating functions (footnote of Sect. 2.2): the plan's band-limits,
    the analysis maps, the synthesis of the oracle's maps and the adjoint against
    the oracle's B-spline transform."""
    seeds = [31, 32]
    f = _maps(L, seeds, real)
    plan = Plan(L, B, J0, batch=len(seeds), real=real, multires=multires, kernel="bspline", **plan_kwargs(prec))
    n_scal, n_wav = wavelet.bandlimits(L, B, J0, multires, "bspline")
    assert plan.N_scal == n_scal and [n for (_, n, _, _) in plan.scales] == n_wav
    fw_d, fs_d = plan.analysis(to_dev_map(f, plan.dtype, real))
    ref = [wavelet.analysis(x, L, B, J0, multires, real, kernel="bspline") for x in f]
    for i, view in enumerate(plan.wavelet_views(fw_d)):
        want = np.stack([r[0][i] for r in ref])
        assert rel_err(from_dev_map(view, real), want) < TOL[prec], "scale %d" % (J0 + i)
    assert rel_err(from_dev_map(fs_d, real), np.stack([r[1] for r in ref])) < TOL[prec]
    fw_in = torch.cat([to_dev_map(np.stack([r[0][i] for r in ref]), plan.dtype, real).reshape(-1)
                       for i in range(len(ref[0][0]))])
    fs_in = to_dev_map(np.stack([r[1] for r in ref]), plan.dtype, real)
    rec = from_dev_map(plan.synthesis(fw_in, fs_in), real)
    assert rel_err(rec, f) < TOL[prec]
    # adjoint of the analysis on random wavelet-space inputs
    gws = [[inputs.random_map((n, 2 * n - 1), 300 * b + i, real) for i, n in enumerate(n_wav)] for b in range(2)]
    gss = [inputs.random_map((n_scal, 2 * n_scal - 1), 97 + b, real) for b in range(2)]
    gw = torch.cat([to_dev_map(np.stack([g[i] for g in gws]), plan.dtype, real).reshape(-1)
                    for i in range(len(n_wav))])
    got = from_dev_map(plan.adjoint(gw, to_dev_map(np.stack(gss), plan.dtype, real)), real)
    want = np.stack([wavelet.analysis_adjoint(gws[b], gss[b], L, B, J0, multires, real, kernel="bspline")
                     for b in range(2)])
    assert rel_err(got, want) < TOL[prec]
    assert plan.status() == 0


def test_plans_of_different_sizes_coexist():
    """A smaller plan created after a larger one must not break the larger one."""
    big = Plan(200, 2, 1, batch=1, real=True, precision="fp32")
    small = Plan(8, 2, 1, batch=1, real=True, precision="fp32")
    for plan, L in ((big, 200), (small, 8), (big, 200)):
        flm = inputs.random_flm(L, 3, True)
        f = from_dev_map(plan.sht_inverse(flm_to_dev(flm[None], plan.dtype)), True)
        assert rel_err(f[0], sht.inverse(flm, L, real=True)) < TOL["fp32"]


@pytest.mark.parametrize("prec,real", [("tf32x3", True), ("tf32x3", False), ("fp32", True)])
def test_autotuned_plan_keeps_parity(prec, real):
    """After s2let_plan_autotune (kernel choice per stage and band-limit, ring-DFT
    block size) the transforms still match the oracle."""
    L = 160
    flm = np.stack([inputs.random_flm(L, s, real) for s in (51, 52)])
    plan = Plan(L, 2, 1, batch=2, real=real, multires=True, precision=prec)
    tuning = plan.autotune()
    assert set(tuning) >= {L, plan.N_scal}
    for n, t in tuning.items():
        assert 32 <= t["fft_threads"] <= 512
        if prec != "tf32x3":
            assert not (t["tc_quad"] or t["tc_anal"] or t["tc_synth"])
    f_ref = np.stack([sht.inverse(x, L, real=real) for x in flm])
    f_gpu = from_dev_map(plan.sht_inverse(flm_to_dev(flm, plan.dtype)), real)
    assert rel_err(f_gpu, f_ref) < TOL[prec]
    g = flm_from_dev(plan.sht_forward(to_dev_map(f_ref, plan.dtype, real)))
    assert rel_err(g, np.stack([sht.forward(x, L) for x in f_ref])) < TOL[prec]
    f = np.stack(f_ref)
    fw_d, fs_d = plan.analysis(to_dev_map(f, plan.dtype, real))
    rec = from_dev_map(plan.synthesis(fw_d, fs_d), real)
    assert rel_err(rec, f) < TOL[prec]
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("L", [4, 8, 23, 32, 33, 50, 158])
def test_mixed_radix_band_limits(L, prec):
    """Band-limits whose ring length P = 2L - 1 factors into 3, 5, 7, 9, 11, 13
    (7, 15, 45, 63, 65, 99, 315) run the mixed-radix ring DFTs (real maps) and
    the FFT form of the theta quadrature: forward and inverse transforms of
    three real maps against the oracle, and a not band-limited map forward."""
    seeds = [61, 62, 63]
    plan = Plan(L, 2, 0, batch=len(seeds), real=True, multires=True, precision=prec)
    flm = np.stack([inputs.random_flm(L, s, True, "cl" if L > 30 else "white") for s in seeds])
    f_ref = np.stack([sht.inverse(x, L, real=True) for x in flm])
    f_gpu = from_dev_map(plan.sht_inverse(flm_to_dev(flm, plan.dtype)), True)
    assert rel_err(f_gpu, f_ref) < TOL[prec]
    g = flm_from_dev(plan.sht_forward(to_dev_map(f_ref, plan.dtype, True)))
    assert rel_err(g, np.stack([sht.forward(x, L) for x in f_ref])) < TOL[prec]
    x = np.stack([inputs.random_map((L, 2 * L - 1), 70 + s) for s in range(len(seeds))])
    g = flm_from_dev(plan.sht_forward(to_dev_map(x, plan.dtype, True)))
    assert rel_err(g, np.stack([sht.forward(v, L) for v in x])) < TOL[prec]
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_mixed_radix_wavelets(prec):
    """L = 158 (P = 315 = 9 x 7 x 5) with multiresolution bands at 4, 8, 32
    (mixed radix) and 16, 64, 128 (Bluestein, dense quadrature): analysis maps,
    synthesis of the oracle's maps, and the adjoint."""
    L, B, J0 = 158, 2, 1
    seeds = [81, 82]
    f = _maps(L, seeds, True)
    plan = Plan(L, B, J0, batch=len(seeds), real=True, multires=True, precision=prec)
    fw_d, fs_d = plan.analysis(to_dev_map(f, plan.dtype, True))
    ref = [wavelet.analysis(x, L, B, J0, True, True) for x in f]
    for i, view in enumerate(plan.wavelet_views(fw_d)):
        assert rel_err(from_dev_map(view, True), np.stack([r[0][i] for r in ref])) < TOL[prec], "scale %d" % (J0 + i)
    assert rel_err(from_dev_map(fs_d, True), np.stack([r[1] for r in ref])) < TOL[prec]
    fw_in = torch.cat([to_dev_map(np.stack([r[0][i] for r in ref]), plan.dtype, True).reshape(-1)
                       for i in range(len(ref[0][0]))])
    rec = from_dev_map(plan.synthesis(fw_in, to_dev_map(np.stack([r[1] for r in ref]), plan.dtype, True)), True)
    assert rel_err(rec, f) < TOL[prec]
    n_scal, n_wav = kernels.bandlimits(L, B, J0, True)
    gws = [[inputs.random_map((n, 2 * n - 1), 400 * b + i) for i, n in enumerate(n_wav)] for b in range(2)]
    gss = [inputs.random_map((n_scal, 2 * n_scal - 1), 57 + b) for b in range(2)]
    gw = torch.cat([to_dev_map(np.stack([g[i] for g in gws]), plan.dtype, True).reshape(-1)
                    for i in range(len(n_wav))])
    got = from_dev_map(plan.adjoint(gw, to_dev_map(np.stack(gss), plan.dtype, True)), True)
    want = np.stack([wavelet.analysis_adjoint(gws[b], gss[b], L, B, J0, True, True) for b in range(2)])
    assert rel_err(got, want) < TOL[prec]
    assert plan.status() == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_fft_quadrature_complex_maps(prec):
    """Complex maps at L = 158: the FFT-form quadrature takes the orders
    |m| > 32 on both sides of the order-major rows, the dense product the
    middle ones (ring DFTs by Bluestein)."""
    L = 158
    flm = np.stack([inputs.random_flm(L, s, False) for s in (91, 92)])
    f_ref = np.stack([sht.inverse(x, L) for x in flm])
    plan = Plan(L, 2, 1, batch=2, real=False, multires=True, precision=prec)
    g = flm_from_dev(plan.sht_forward(to_dev_map(f_ref, plan.dtype, False)))
    assert rel_err(g, flm) < TOL[prec]
    x = np.stack([inputs.random_map((L, 2 * L - 1), 95 + s, False) for s in range(2)])
    g = flm_from_dev(plan.sht_forward(to_dev_map(x, plan.dtype, False)))
    assert rel_err(g, np.stack([sht.forward(v, L) for v in x])) < TOL[prec]
    assert plan.status() == 0

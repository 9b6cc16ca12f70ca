"""Precomputed Legendre tables of the TF32X3 plans: the tensor-core Legendre
kernels that stream them against the oracle and against the same plan with
the float-float recurrence (S2LET_LEG_RECURRENCE), at band-limits whose tables
have ragged edges (orders with a last degree tile of a few degrees, ring
blocks past N, polar ring blocks with no stored block), real and complex maps,
and two batch tiles; plus the size bookkeeping."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sht, wavelet  # noqa: E402
from paper_1211_1680_gb300 import inputs  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402
from tests.gpu_util import TOL, flm_from_dev, flm_to_dev, from_dev_map, rel_err, to_dev_map  # noqa: E402


def _table_bytes_bound(N):
    """Every degree block of every (order, ring block) plus the zero block, 4 KB each,
    in two copies (rows = degrees for the analysis, rows = rings for the synthesis)."""
    nkr = (N + 31) // 32
    return 2 * 4096 * (1 + nkr * sum((N - m + 31) // 32 for m in range(N)))


@pytest.mark.parametrize("real,nb", [(True, 3), (False, 3), (True, 70), (False, 35)])
@pytest.mark.parametrize("L", [45, 161])
def test_tables_against_oracle_and_recurrence(L, real, nb):
    """Forward and inverse transforms on the tables against the oracle (TF32X3
    tolerance) and against the recurrence kernels; 70 real / 35 complex maps
    take two batch tiles."""
    seeds = list(range(500, 500 + nb))
    flm = np.stack([inputs.random_flm(L, s, real, "white") for s in seeds])
    tab = Plan(L, 2, 0, batch=nb, real=real, precision="tf32x3")
    rec = Plan(L, 2, 0, batch=nb, real=real, precision="tf32x3", leg_recurrence=True)
    assert tab.table_bytes(L) > 0 and rec.table_bytes() == 0
    assert tab.tuning()[L]["table_anal"] and tab.tuning()[L]["table_synth"]
    assert not rec.tuning()[L]["table_anal"] and not rec.tuning()[L]["table_synth"]
    sub = [0, nb // 2, nb - 1]                      # the oracle on three maps of the batch
    f_ref = np.stack([sht.inverse(flm[b], L, real=real) for b in sub])
    x = flm_to_dev(flm, tab.dtype)
    f_tab = from_dev_map(tab.sht_inverse(x), real)
    f_rec = from_dev_map(rec.sht_inverse(x), real)
    assert rel_err(f_tab[sub], f_ref) < TOL["tf32x3"]
    assert rel_err(f_tab, f_rec) < 2e-6
    fd = to_dev_map(f_tab, tab.dtype, real)
    g_tab = flm_from_dev(tab.sht_forward(fd))
    g_rec = flm_from_dev(rec.sht_forward(fd))
    ref = np.stack([sht.forward(f_tab[b], L) for b in sub])
    assert rel_err(g_tab[sub], ref) < TOL["tf32x3"]
    assert rel_err(g_tab, g_rec) < 2e-6
    assert tab.status() == 0 and rec.status() == 0


@pytest.mark.parametrize("real", [True, False])
def test_tables_column_scales(real):
    """The FP16 operands of the table kernels are scaled per column (map, order):
    maps of magnitude 1e-30, 1 and 1e30 and an all-zero map in one batch
    transform like the unit map scaled (each within the tolerance of its own
    magnitude; the zero map to exact zeros)."""
    L = 72
    base = inputs.random_flm(L, 700, real, "white")
    mags = [1e-30, 1.0, 1e30]
    flm = np.stack([base * s for s in mags] + [np.zeros_like(base)])
    plan = Plan(L, 2, 0, batch=4, real=real, precision="tf32x3")
    assert plan.tuning()[L]["table_anal"] and plan.tuning()[L]["table_synth"]
    f = from_dev_map(plan.sht_inverse(flm_to_dev(flm, plan.dtype)), real)
    f_ref = sht.inverse(base, L, real=real)
    for b, s in enumerate(mags):
        assert rel_err(f[b] / s, f_ref) < TOL["tf32x3"], "map %d" % b
    assert np.all(f[3] == 0)
    g = flm_from_dev(plan.sht_forward(to_dev_map(f, plan.dtype, real)))
    g_ref = sht.forward(f[1], L)
    for b, s in enumerate(mags):
        assert rel_err(g[b] / s, g_ref) < TOL["tf32x3"], "map %d" % b
    assert np.all(g[3] == 0)
    assert plan.status() == 0


@pytest.mark.parametrize("real", [True, False])
def test_tables_wavelets_accumulate(real):
    """Wavelet synthesis sums the analysis of every scale into one set of
    coefficients (the accumulating path of the table kernel); analysis and
    synthesis against the oracle, multiresolution band-limits 8 .. 96."""
    L, B, J0 = 96, 2, 2
    seeds = [601, 602]
    f = np.stack([sht.inverse(inputs.random_flm(L, s, real, "white"), L, real=real) for s in seeds])
    plan = Plan(L, B, J0, batch=len(seeds), real=real, multires=True, precision="tf32x3")
    assert plan.table_bytes() > 0
    fw, fs = plan.analysis(to_dev_map(f, plan.dtype, real))
    ref = [wavelet.analysis(x, L, B, J0, True, real) for x in f]
    assert rel_err(from_dev_map(fs, real), np.stack([r[1] for r in ref])) < TOL["tf32x3"]
    for i, v in enumerate(plan.wavelet_views(fw)):
        assert rel_err(from_dev_map(v, real), np.stack([r[0][i] for r in ref])) < TOL["tf32x3"], "scale %d" % i
    rec = from_dev_map(plan.synthesis(fw, fs), real)
    assert rel_err(rec, f) < TOL["tf32x3"]
    assert plan.status() == 0


@pytest.mark.parametrize("real,nb", [(True, 70), (False, 35)])
def test_two_map_streams_two_batch_tiles(real, nb):
    """The wavelet scales 5 and 6 of L = 64 (B = 2) share the band-limit 64, so the
    analysis runs their syntheses as one two-map launch on one table stream and the
    synthesis their analyses likewise; with 70 real (35 complex) maps both run two
    batch tiles.  Maps of both tiles against the oracle."""
    L, B, J0 = 64, 2, 2
    seeds = list(range(800, 800 + nb))
    sub = [0, nb // 2 + 3, nb - 1]
    f = np.stack([sht.inverse(inputs.random_flm(L, s, real, "white"), L, real=real) for s in seeds])
    plan = Plan(L, B, J0, batch=nb, real=real, multires=True, precision="tf32x3")
    assert plan.tuning()[L]["table_anal"] and plan.tuning()[L]["table_synth"]
    assert [n for (_, n, _, _) in plan.scales][-2:] == [L, L]
    fw, fs = plan.analysis(to_dev_map(f, plan.dtype, real))
    views = plan.wavelet_views(fw)
    for b in sub:
        ref_w, ref_s = wavelet.analysis(f[b], L, B, J0, True, real)
        for i, v in enumerate(views):
            assert rel_err(from_dev_map(v, real)[b], ref_w[i]) < TOL["tf32x3"], (b, i)
        assert rel_err(from_dev_map(fs, real)[b], ref_s) < TOL["tf32x3"], b
    rec = from_dev_map(plan.synthesis(fw, fs), real)
    assert rel_err(rec[sub], f[sub]) < TOL["tf32x3"]
    assert rel_err(rec, f) < TOL["tf32x3"]
    assert plan.status() == 0


def test_table_bytes_per_band_limit():
    """Per band-limit sizes add up to the total, stay within every-block bound,
    and leave out polar blocks below 2^-100 at N = 256."""
    L = 256
    plan = Plan(L, 2, 2, batch=1, real=True, multires=True, precision="tf32x3")
    ns = sorted({L, plan.N_scal} | {s[1] for s in plan.scales})
    per = {n: plan.table_bytes(n) for n in ns}
    assert sum(per.values()) == plan.table_bytes()
    for n in ns:
        assert 0 < per[n] <= _table_bytes_bound(n)
    assert per[L] < _table_bytes_bound(L)

"""Band-limit L = 4096, the top of the range the MW sampling theorem is stable
to (Sect. 2.1): one real map, B = 2, J_min = 2, multiresolution, in the FP32 and
TF32X3 plans.  The input holds the full degree range of a few orders (and their
negatives, for a real map), so that the oracle's inverse restricted to those
orders gives the map exactly without the cost of a full L = 4096 transform.
Checked against the oracle: every harmonic coefficient of the forward
transform, the wavelet maps of the finest scales on sampled rings (the direct
sum of Eq. wav2), and the reconstruction of the map."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sht, wavelet  # noqa: E402
from paper_1211_1680_gb300 import inputs  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402
from tests.gpu_util import TOL, flm_from_dev, rel_err  # noqa: E402

L, B, J0 = 4096, 2, 2
ORDERS = [0, 1, 2, 7, 100, 1023, 2500, 4095]


@pytest.fixture(scope="module")
def oracle_case():
    flm = inputs.random_flm(L, 4096, True, "cl")
    l_of = np.repeat(np.arange(L), 2 * np.arange(L) + 1)
    m_of = np.arange(L * L) - l_of * l_of - l_of
    flm[~np.isin(np.abs(m_of), ORDERS)] = 0.0
    orders = sorted(set(ORDERS) | {-m for m in ORDERS})
    x = sht.inverse(flm, L, real=True, orders=orders)
    return flm, x, l_of


@pytest.mark.parametrize("prec", ["tf32x3", "fp32"])
def test_band_limit_4096(prec, oracle_case):
    flm, x, l_of = oracle_case
    plan = Plan(L, B, J0, batch=1, real=True, multires=True, precision=prec)
    xd = torch.from_numpy(x[None].astype(np.float32)).cuda()
    g = flm_from_dev(plan.sht_forward(xd))[0]
    assert rel_err(g, flm) < TOL[prec], "forward transform"
    fw, fs = plan.analysis(xd)
    rec = plan.synthesis(fw, fs)
    torch.cuda.synchronize()
    assert rel_err(rec[0].double().cpu().numpy(), x) < TOL[prec], "reconstruction"
    phi, psi = wavelet.tables(L, B, J0)
    norm = np.sqrt(4 * np.pi / (2 * l_of + 1))
    views = plan.wavelet_views(fw)
    for (j, n, _, _), kern, v in zip(plan.scales, psi, views):
        if n < L:
            continue                                     # the finest scales, at the full band-limit
        rings = [0, 1, n // 4, n // 2, n - 2, n - 1]
        ref = sht.inverse_at((norm * flm * kern[l_of])[:n * n], n, rings, np.arange(2 * n - 1)).real
        got = v[0].double().cpu().numpy()[rings]
        assert np.max(np.abs(got - ref)) / v[0].double().abs().max().item() < TOL[prec], "scale %d" % j
    assert plan.status() == 0

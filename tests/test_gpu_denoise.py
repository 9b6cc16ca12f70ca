"""GPU: wavelet denoising by hard thresholding (Sect. 4.3) through the C ABI
against the oracle: the per-scale noise standard deviations (Eq. noisemodel),
the threshold decisions (Eq. threshold; bit-exact, taken in the plan's
precision on both sides) and the denoised map."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sht, wavelet  # noqa: E402
from paper_1211_1680_gb300 import inputs  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402
from tests.gpu_util import TOL, from_dev_map, rel_err, to_dev_map  # noqa: E402
from tests.test_oracle_wavelet import spot_signal  # noqa: E402


@pytest.mark.parametrize("L,B,J0,kernel", [(32, 2, 0, "sd"), (130, 3, 1, "sd"), (64, 2, 1, "bspline")])
def test_noise_std_matches_oracle(L, B, J0, kernel):
    plan = Plan(L, B, J0, batch=1, real=True, precision="fp32", kernel=kernel)
    s_phi, s_j = wavelet.noise_std(L, B, J0, kernel)
    assert plan.noise_std(-1) == pytest.approx(s_phi, rel=1e-12, abs=1e-15)
    for j, s in zip(range(J0, plan.J + 1), s_j):
        assert plan.noise_std(j) == pytest.approx(s, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("prec,real", [("fp32", True), ("fp32", False), ("fp64", True), ("fp64", False),
                                       ("tf32x3", True)])
def test_threshold_decisions_bit_exact(prec, real):
    """Random wavelet maps straddling each scale's threshold: the kernel's output
    equals the same test made on the host in the plan's precision."""
    L, B, J0, sigma, nsig = 64, 2, 1, 0.37, 3.0
    plan = Plan(L, B, J0, batch=3, real=real, multires=True, precision=prec)
    dt = np.float64 if prec == "fp64" else np.float32
    maps = []
    for i, (j, n, _, _) in enumerate(plan.scales):
        T = nsig * sigma * plan.noise_std(j)
        maps.append(T * 2.0 * np.stack([inputs.random_map((n, 2 * n - 1), 40 * i + b, real) for b in range(3)]))
    fw = torch.cat([to_dev_map(m, plan.dtype, real).reshape(-1) for m in maps])
    plan.threshold(fw, sigma, nsig)
    got = [from_dev_map(v, real) for v in plan.wavelet_views(fw)]
    zeroed = 0
    for (j, n, _, _), m, g in zip(plan.scales, maps, got):
        T = dt(nsig * sigma * plan.noise_std(j))
        if real:
            x = m.astype(dt)
            want = np.where(np.abs(x) < T, dt(0), x)
        else:
            re, im = m.real.astype(dt), m.imag.astype(dt)
            keep = ~((re * re + im * im) < T * T)
            want = np.where(keep, re, dt(0)) + 1j * np.where(keep, im, dt(0))
        assert np.array_equal(np.asarray(g), np.asarray(want)), "scale %d" % j
        zeroed += int(np.sum(np.asarray(want) == 0))
    # the thresholds are active: |2 T N(0,1)| < T for 38% of real samples, and
    # |2 T (N(0,1) + i N(0,1))| < T for 1 - exp(-1/8) = 11.8% of complex ones
    assert zeroed > (0.3 if real else 0.09) * sum(m.size for m in maps)
    assert plan.status() == 0


def _noisy(L, snr_db, seed):
    s = spot_signal(L)
    energy = float(np.sum(np.abs(sht.forward(s, L)) ** 2))
    sigma = math.sqrt(energy / (L * L) / 10 ** (snr_db / 10))
    return s, s + sht.inverse(sigma * inputs.random_flm(L, seed, True, "white"), L, real=True), sigma


def test_denoise_matches_oracle_fp64():
    L, B, J0 = 32, 2, 0
    s, y, sigma = _noisy(L, 5.0, 8)
    plan = Plan(L, B, J0, batch=1, real=True, multires=True, precision="fp64")
    d = from_dev_map(plan.denoise(to_dev_map(y[None], plan.dtype, True), sigma), True)[0]
    want = wavelet.denoise(y, sigma, L, B, J0, multires=True, real=True)
    assert rel_err(d, want) < TOL["fp64"]
    assert wavelet.snr_db(s, d, L) > wavelet.snr_db(s, y, L) + 5.0


@pytest.mark.parametrize("kernel", ["sd", "bspline"])
def test_denoise_raises_snr_tf32x3(kernel):
    """The default precision: the SNR gain of the oracle's denoising is reproduced
    (individual threshold decisions may differ near T^j at this precision)."""
    L, B, J0 = 96, 2, 1
    s, y, sigma = _noisy(L, 5.0, 11)
    plan = Plan(L, B, J0, batch=1, real=True, multires=True, precision="tf32x3", kernel=kernel)
    d = from_dev_map(plan.denoise(to_dev_map(y[None], plan.dtype, True), sigma), True)[0]
    want = wavelet.denoise(y, sigma, L, B, J0, multires=True, real=True, kernel=kernel)
    gain = wavelet.snr_db(s, d, L) - wavelet.snr_db(s, y, L)
    gain_oracle = wavelet.snr_db(s, want, L) - wavelet.snr_db(s, y, L)
    assert gain > 3.0 and abs(gain - gain_oracle) < 0.05
    assert plan.status() == 0

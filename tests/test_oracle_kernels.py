"""Pins for the oracle's wavelet kernels (Sect. 2.2) and band-limits (Sect. 3.1)."""
import math
import os

import numpy as np
import pytest

from oracle import kernels, wavelet

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_bump_values_and_support():
    assert kernels.s(0.0) == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert kernels.s(1.0) == 0.0 and kernels.s(-1.0) == 0.0 and kernels.s(1.5) == 0.0
    # s_lambda has support [1/lambda, 1] and peaks at its midpoint
    for lam in (2.0, 3.0):
        assert kernels.s_lambda(1.0 / lam, lam) == 0.0
        assert kernels.s_lambda(1.0, lam) == 0.0
        mid = 0.5 * (1.0 / lam + 1.0)
        assert kernels.s_lambda(mid, lam) == pytest.approx(math.exp(-1.0), rel=1e-14)


@pytest.mark.parametrize("lam", [2.0, 3.0, 1.7])
def test_k_endpoints_and_monotone(lam):
    assert kernels.k_lambda(1.0 / lam, lam) == 1.0
    assert kernels.k_lambda(0.0, lam) == 1.0
    assert kernels.k_lambda(1.0, lam) == 0.0
    ts = np.linspace(1.0 / lam, 1.0, 41)
    ks = [kernels.k_lambda(t, lam) for t in ts]
    assert all(a >= b for a, b in zip(ks, ks[1:]))


def test_k_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30

    def s_mp(t):
        return mpmath.e ** (-1 / (1 - t * t)) if -1 < t < 1 else mpmath.mpf(0)

    for lam in (2, 3):
        def f(u):
            x = 2 * mpmath.mpf(lam) / (lam - 1) * (u - mpmath.mpf(1) / lam) - 1
            return s_mp(x) ** 2 / u
        den = mpmath.quad(f, [mpmath.mpf(1) / lam, 1])
        for t in (0.55, 0.6, 0.75, 0.9, 0.99) if lam == 2 else (0.4, 0.5, 0.7, 0.95):
            ref = mpmath.quad(f, [t, 1]) / den
            assert kernels.k_lambda(t, lam) == pytest.approx(float(ref), abs=1e-13)


@pytest.mark.parametrize("L,B,J0", [(32, 2, 0), (128, 3, 2), (512, 2, 2), (100, 3, 1), (65, 2, 5)])
def test_admissibility_identity(L, B, J0):
    """Eq. (identity): 4 pi/(2l+1) (|Phi_l0|^2 + sum_j |Psi^j_l0|^2) = 1 for all l < L."""
    phi, psi = wavelet.tables(L, B, J0)
    l = np.arange(L)
    total = 4 * np.pi / (2 * l + 1) * (phi ** 2 + sum(p ** 2 for p in psi))
    assert np.max(np.abs(total - 1.0)) < 1e-14


@pytest.mark.parametrize("L,B,J0", [(128, 3, 2), (256, 2, 1)])
def test_wavelet_and_scaling_support(L, B, J0):
    """Psi^j has support in (lambda^{j-1}, lambda^{j+1}); Phi is zero for l >= lambda^J0."""
    phi, psi = wavelet.tables(L, B, J0)
    l = np.arange(L)
    assert np.all(phi[l >= B ** J0] == 0.0)
    assert np.all(phi[l < B ** (J0 - 1)] > 0.0) if J0 >= 1 else True
    for j, p in zip(range(J0, J0 + len(psi)), psi):
        outside = (l <= B ** (j - 1)) | (l >= B ** (j + 1))
        assert np.all(p[outside] == 0.0)
        assert np.all(p[~outside] >= 0.0)


def test_jmax_and_figure_parameters():
    vals = {}
    with open(os.path.join(GOLDEN, "fig_kernels_scales.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = [int(x) for x in v]
    L, lam, J0 = vals["L"][0], vals["lambda"][0], vals["J0"][0]
    J = kernels.jmax(L, lam)
    assert list(range(J0, J + 1)) == vals["scales"]
    assert J - J0 + 3 == vals["n_sht"][0]
    assert (L - 1) * (2 * L - 1) + 1 == vals["n_samples"][0]
    # J = ceil(log_lambda(L-1)), including the exact power case
    for L_, B_ in [(3, 2), (9, 2), (10, 3), (28, 3), (2049, 2), (2048, 2), (4096, 2)]:
        assert kernels.jmax(L_, B_) == math.ceil(round(math.log(L_ - 1, B_), 12))


def test_bandlimits():
    assert kernels.bandlimits(512, 2, 2, True) == (4, [8, 16, 32, 64, 128, 256, 512, 512])
    assert kernels.bandlimits(32, 2, 0, False) == (32, [32] * 6)
    assert kernels.bandlimits(2048, 3, 1, True) == (3, [9, 27, 81, 243, 729, 2048, 2048])
    with pytest.raises(ValueError):
        kernels.bandlimits(32, 2, 5, True)   # J0 must be < J = 5


def test_kappa_relative_accuracy_near_support_edges():
    """kappa(t) where k(t/lambda) and k(t) are both within 1e-16 of 1 (t just
    above 1/lambda), and elsewhere, against mpmath at 40 digits (kappa =
    8.8e-9 at t = 65/128, lambda = 2; computed as a difference of two ratios
    it would round to 0)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for lam in (2, 3):
        def s_mp(x):
            return mpmath.e ** (-1 / (1 - x * x)) if -1 < x < 1 else mpmath.mpf(0)

        def f(u):
            x = 2 * mpmath.mpf(lam) / (lam - 1) * (u - mpmath.mpf(1) / lam) - 1
            return s_mp(x) ** 2 / u
        den = mpmath.quad(f, [mpmath.mpf(1) / lam, 1])
        for t in (1.0 / lam + 0.004, 65.0 / 128 if lam == 2 else 0.34, 1.0 / lam + 0.05, 0.9, 0.99,
                  1.3, lam * 0.99):
            lo, hi = max(t / lam, 1.0 / lam), min(t, 1.0)
            ref = float(mpmath.sqrt(mpmath.quad(f, [lo, hi]) / den))
            got = kernels.kappa_lambda(t, lam)
            assert got > 0.0
            # absolute accuracy at the FP64 level everywhere, relative where kappa > 1e-12
            assert abs(got - ref) < 2e-16 + (1e-11 * ref if ref > 1e-12 else 0.0)

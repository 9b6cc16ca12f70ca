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


# ---------------------------------------------------------------- B-spline family (footnote of Sect. 2.2)
def test_bspline3_values_and_partition_of_unity():
    """The cubic B-spline: B_3(0) = 2/3, B_3(+-1) = 1/6, B_3(+-1/2) = 23/48, zero for
    |x| >= 2, and its integer translates sum to one (the textbook properties, which
    any dropped term or wrong coefficient of the five-term sum breaks)."""
    B3 = kernels.bspline3
    assert B3(0.0) == pytest.approx(2.0 / 3.0, abs=1e-15)
    assert B3(1.0) == pytest.approx(1.0 / 6.0, abs=1e-15) and B3(-1.0) == pytest.approx(1.0 / 6.0, abs=1e-15)
    assert B3(0.5) == pytest.approx(23.0 / 48.0, abs=1e-15) and B3(-0.5) == pytest.approx(23.0 / 48.0, abs=1e-15)
    for x in (2.0, -2.0, 2.5, -3.7):
        assert abs(B3(x)) < 1e-15
    for x in np.linspace(-0.5, 0.5, 11):
        assert sum(B3(x - k) for k in range(-3, 4)) == pytest.approx(1.0, abs=1e-14)
    # piecewise form on [0, 1] and [1, 2]
    for x in np.linspace(0.0, 1.0, 9):
        assert B3(x) == pytest.approx(2.0 / 3.0 - x * x + x ** 3 / 2.0, abs=1e-14)
    for x in np.linspace(1.0, 2.0, 9):
        assert B3(x) == pytest.approx((2.0 - x) ** 3 / 6.0, abs=1e-14)


@pytest.mark.parametrize("L,B,J0", [(32, 2, 0), (128, 3, 2), (256, 2, 1), (100, 3, 1)])
def test_bspline_admissibility(L, B, J0):
    """With the finest scale taking the remainder, the squared B-spline kernels of
    all scales and the scaling function sum to one for every l < L (exact
    reconstruction, Eq. identity)."""
    phi, psi = wavelet.tables(L, B, J0, "bspline")
    l = np.arange(L)
    total = 4 * np.pi / (2 * l + 1) * (phi ** 2 + sum(p ** 2 for p in psi))
    assert np.max(np.abs(total - 1.0)) < 1e-14


@pytest.mark.parametrize("L,B,J0", [(128, 3, 2), (256, 2, 1), (2048, 2, 2), (500, 3, 0)])
def test_bspline_support_and_bandlimits(L, B, J0):
    """The j-th B-spline filter (j < J) has support [0, L / lambda^(J-j-2)) (footnote of
    Sect. 2.2 and Sect. 3.1); the scaling function vanishes from L / lambda^(J-J0-1) on;
    the multiresolution band-limits are the (capped) ends of these supports."""
    J = kernels.jmax(L, B)
    phi, psi = wavelet.tables(L, B, J0, "bspline")
    l = np.arange(L)
    for j, p in zip(range(J0, J + 1), psi):
        end = L / B ** (J - j - 2)
        if j < J:
            assert np.all(p[l >= end] == 0.0)
            assert np.all(p[(l > 0) & (l < end)] > 0.0)
        assert p[0] == 0.0                          # no scale sees the monopole but the scaling function
    assert np.all(phi[l >= L / B ** (J - J0 - 1)] == 0.0)
    assert np.all(phi[l < L / B ** (J - J0 - 1)] > 0.0)
    n_scal, n_wav = wavelet.bandlimits(L, B, J0, True, "bspline")
    assert n_scal == min(L, math.ceil(L / B ** (J - J0 - 1)))
    assert n_wav == [min(L, math.ceil(L / B ** (J - j - 2))) if J - j - 2 > 0 else L for j in range(J0, J + 1)]
    # every kernel vanishes at and beyond its band-limit
    assert np.all(phi[n_scal:] == 0.0)
    for p, n in zip(psi, n_wav):
        assert np.all(p[n:] == 0.0)
    # B-spline scales are at least as wide as the scale-discretised ones (Sect. 3.1)
    _, n_sd = kernels.bandlimits(L, B, J0, True)
    assert all(a >= b for a, b in zip(n_wav, n_sd))


def test_bspline_k_shape():
    """k(t) = 3/2 B_3(2 t lambda^(J-1) / L): 1 at t = 0, 0 from t = L / lambda^(J-1) on,
    strictly decreasing in between."""
    L, lam = 256, 2
    J = kernels.jmax(L, lam)
    t_end = L / lam ** (J - 1)
    assert kernels.k_bspline(0.0, lam, L, J) == pytest.approx(1.0, abs=1e-15)
    assert kernels.k_bspline(t_end, lam, L, J) == 0.0
    ts = np.linspace(0.0, t_end, 33)
    ks = [kernels.k_bspline(t, lam, L, J) for t in ts]
    assert all(a > b for a, b in zip(ks[:-1], ks[1:]))


@pytest.mark.parametrize("L,B,J0", [(128, 3, 2), (256, 2, 1), (1024, 2, 2)])
def test_bspline_peaks_match_scale_discretised(L, B, J0):
    """The footnote of Sect. 2.2 chooses k so that the j-th B-spline filter peaks at
    about the scale of the j-th scale-discretised filter: the peak degrees agree
    within 30% at every scale (a wrong power of lambda in k would move them by a
    factor lambda)."""
    l = np.arange(L)
    norm = np.sqrt((2 * l + 1) / (4 * np.pi))
    _, psi_sd = wavelet.tables(L, B, J0, "sd")
    _, psi_bs = wavelet.tables(L, B, J0, "bspline")
    for a, b in zip(psi_sd, psi_bs):
        pa, pb = int(np.argmax(a / norm)), int(np.argmax(b / norm))
        assert 0.8 <= pb / max(pa, 1) <= 1.3

"""Pins for the oracle's Legendre functions and MW spherical harmonic transforms
(Sect. 2.1).  Each check compares against something other than the oracle:
closed forms, scipy's spherical harmonics, mpmath, an independent Gauss-Legendre
quadrature, or analytic maps with known coefficients."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import sht
from paper_1211_1680_gb300 import inputs


def _lam(m, N, theta):
    x = math.cos(theta)
    return sht.legendre_column(m, N, math.sin(theta), 1.0 if x >= 0 else -1.0, 1.0 - abs(x))


@pytest.mark.parametrize("theta", [0.1, 0.7, 1.3, 2.0, 3.0])
def test_legendre_closed_forms(theta):
    c, s = math.cos(theta), math.sin(theta)
    pi = math.pi
    ref = {
        (0, 0): 1 / math.sqrt(4 * pi),
        (1, 0): math.sqrt(3 / (4 * pi)) * c,
        (1, 1): -math.sqrt(3 / (8 * pi)) * s,
        (2, 0): math.sqrt(5 / (4 * pi)) * (3 * c * c - 1) / 2,
        (2, 1): -math.sqrt(15 / (8 * pi)) * s * c,
        (2, 2): math.sqrt(15 / (32 * pi)) * s * s,
    }
    for (l, m), v in ref.items():
        assert _lam(m, 3, theta)[l - m] == pytest.approx(v, abs=1e-15)


def test_legendre_against_scipy():
    """Normalisation and Condon-Shortley phase: Y_lm(theta, 0) from scipy."""
    for theta in (0.05, 0.9, 1.6, 2.5, 3.1):
        for m in (0, 1, 2, 5, 17, 30):
            col = _lam(m, 61, theta)
            for l in range(m, 61, 7):
                y = special.sph_harm_y(l, m, theta, 0.0)
                assert col[l - m] == pytest.approx(y.real, abs=5e-13)


def test_legendre_high_degree_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    N = 512
    P = 2 * N - 1
    for t in (0, 3, 200, 508, 510):
        col0 = sht.legendre_at(0, N, t)
        col1 = sht.legendre_at(1, N, t)
        th = mpmath.pi * (2 * t + 1) / P
        for l in (1, 64, 300, 511):
            r0 = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi)) * mpmath.legendre(l, mpmath.cos(th))
            r1 = (mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi) / (l * (l + 1)))
                  * mpmath.legenp(l, 1, mpmath.cos(th), type=2))
            assert col0[l] == pytest.approx(float(r0), abs=1e-11)
            assert col1[l - 1] == pytest.approx(float(r1), abs=1e-11)


def test_sectoral_beyond_fp64_range():
    """At L = 2048 near the pole lambda_mm is ~1e-6000: the oracle carries it as
    mantissa * 2^exponent.  Pin log2|lambda_mm| and its sign against the closed
    form sqrt((2m+1)/(4 pi) (2m)!/(4^m m!^2)) sin^m(theta) (via lgamma)."""
    N = 2048
    s, sg, y = sht.sin_cos_theta(N, [0, 5])
    for ti in range(2):
        for m in (1000, 2000, 2047):
            val, f, e = sht.legendre_column_x(m, N, s[ti], sg[ti], y[ti])
            log2_ref = (0.5 * math.log2((2 * m + 1) / (4 * math.pi))
                        + 0.5 * (math.lgamma(2 * m + 1) - 2 * math.lgamma(m + 1) - m * math.log(4))
                        / math.log(2) + m * math.log2(s[ti]))
            log2_got = math.log2(abs(f[0])) + e[0]
            assert log2_got == pytest.approx(log2_ref, rel=1e-12, abs=1e-9)
            assert np.sign(f[0]) == (-1) ** m
            assert val[0] == 0.0            # far below the FP64 range


def test_orthonormality_brute_force():
    """2 pi int_0^pi lambda_lm lambda_l'm sin(theta) dtheta = delta_ll' by a
    Gauss-Legendre rule in cos(theta) (independent of the MW quadrature)."""
    L = 16
    x, w = np.polynomial.legendre.leggauss(40)
    for m in range(0, L):
        cols = np.array([sht.legendre_column(m, L, math.sqrt(1 - xi * xi),
                                             1.0 if xi >= 0 else -1.0, 1.0 - abs(xi))
                         for xi in x])                       # [node, l]
        gram = 2 * math.pi * (cols * w[:, None]).T @ cols
        assert np.max(np.abs(gram - np.eye(L - m))) < 2e-13   # y = 1-|x| from a rounded node


def test_weights_closed_form():
    for p in range(-9, 10):
        re, _ = integrate.quad(lambda t: math.cos(p * t) * math.sin(t), 0, math.pi,
                               epsabs=1e-14, epsrel=1e-13)
        im, _ = integrate.quad(lambda t: math.sin(p * t) * math.sin(t), 0, math.pi,
                               epsabs=1e-14, epsrel=1e-13)
        assert sht.weights(p) == pytest.approx(re + 1j * im, abs=1e-14)


def _grid(N):
    th = sht.thetas(N)
    ph = sht.phis(N)
    return np.meshgrid(th, ph, indexing="ij")


def test_forward_of_analytic_maps():
    """Maps with known coefficients: 1 -> sqrt(4 pi) Y_00; cos(theta) ->
    sqrt(4 pi/3) Y_10; sin(theta) cos(phi) -> sqrt(2 pi/3)(Y_{1,-1} - Y_11)."""
    N = 6
    th, ph = _grid(N)
    cases = [
        (np.ones_like(th), {(0, 0): math.sqrt(4 * math.pi)}),
        (np.cos(th), {(1, 0): math.sqrt(4 * math.pi / 3)}),
        (np.sin(th) * np.cos(ph), {(1, -1): math.sqrt(2 * math.pi / 3), (1, 1): -math.sqrt(2 * math.pi / 3)}),
    ]
    for f, ref in cases:
        got = sht.forward(f, N)
        want = np.zeros(N * N, complex)
        for (l, m), v in ref.items():
            want[l * l + l + m] = v
        assert np.max(np.abs(got - want)) < 1e-14


def test_forward_against_scipy_quadrature():
    """f = a band-limited polynomial in (x, y, z); its coefficients by a
    Gauss-Legendre x uniform-phi rule with scipy's Y_lm, against the MW forward."""
    N = 8
    def f(theta, phi):
        x, y, z = np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)
        return 0.3 + x * y * z - 2 * z ** 3 + x ** 4 * y ** 2 + 0.5j * (y ** 5 - x * z ** 6)
    xg, wg = np.polynomial.legendre.leggauss(2 * N)
    tg = np.arccos(xg)
    pg = 2 * np.pi * np.arange(2 * N + 1) / (2 * N + 1)
    T, Pp = np.meshgrid(tg, pg, indexing="ij")
    fv = f(T, Pp)
    ref = np.zeros(N * N, complex)
    for l in range(N):
        for m in range(-l, l + 1):
            Y = special.sph_harm_y(l, m, T, Pp)
            ref[l * l + l + m] = np.sum(wg[:, None] * fv * np.conj(Y)) * 2 * np.pi / (2 * N + 1)
    th, ph = _grid(N)
    got = sht.forward(f(th, ph), N)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_inverse_against_scipy():
    N = 12
    flm = inputs.random_flm(N, 3, real=False)
    th, ph = _grid(N)
    ref = np.zeros(th.shape, complex)
    for l in range(N):
        for m in range(-l, l + 1):
            ref += flm[l * l + l + m] * special.sph_harm_y(l, m, th, ph)
    assert np.max(np.abs(sht.inverse(flm, N) - ref)) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4, 7, 16, 33, 64, 128])
def test_round_trip(N):
    """Exactness of the MW quadrature for band-limited maps (Sect. 2.1)."""
    flm = inputs.random_flm(N, 100 + N, real=False)
    err = np.max(np.abs(sht.forward(sht.inverse(flm, N), N) - flm))
    assert err < 3e-15 * max(N, 4)


def test_real_map_symmetry():
    N = 20
    f = inputs.random_map((N, 2 * N - 1), 5)        # any real samples
    flm = sht.forward(f, N)
    for l in range(N):
        for m in range(1, l + 1):
            assert flm[l * l + l - m] == pytest.approx((-1) ** m * np.conj(flm[l * l + l + m]), abs=1e-14)


def test_forward_m_matches_forward():
    N = 24
    f = sht.inverse(inputs.random_flm(N, 9, real=False), N)
    full = sht.forward(f, N)
    for m in (-23, -4, 0, 1, 11, 23):
        l = np.arange(abs(m), N)
        assert np.max(np.abs(sht.forward_m(f, N, m) - full[l * l + l + m])) < 1e-14


@pytest.mark.parametrize("N", [1, 2, 5, 12])
def test_transform_adjoints(N):
    """<A x, y> = <x, A^H y> for the inverse and forward transforms."""
    x = inputs.random_map((N * N,), 21, real=False)
    g = inputs.random_map((N, 2 * N - 1), 22, real=False)
    lhs = np.vdot(g, sht.inverse(x, N))
    rhs = np.vdot(sht.inverse_adjoint(g, N), x)
    assert lhs == pytest.approx(rhs, rel=1e-13)
    lhs = np.vdot(x, sht.forward(g, N))
    rhs = np.vdot(sht.forward_adjoint(x, N), g)
    assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("N", [1, 7, 33])
def test_inverse_at_matches_full_grid(N):
    """inverse_at (the checker of the full-size GPU maps) selects the right rings
    and longitudes: it equals the full inverse transform on the same grid points,
    with rings and longitudes scattered, repeated and out of order."""
    flm = inputs.random_flm(N, 70 + N, real=False)
    full = sht.inverse(flm, N)
    rng = np.random.default_rng(N)
    ts = rng.integers(0, N, size=min(N, 5) + 1)
    ps = rng.integers(0, 2 * N - 1, size=min(2 * N - 1, 9) + 1)
    got = sht.inverse_at(flm, N, ts, ps)
    assert got.shape == (len(ts), len(ps))
    assert np.max(np.abs(got - full[ts][:, ps])) < 1e-13


def test_inverse_at_against_scipy():
    """inverse_at at scattered grid points against the direct sum of scipy's Y_lm."""
    N = 14
    flm = inputs.random_flm(N, 5, real=False)
    ts, ps = np.array([13, 0, 6, 6, 2]), np.array([26, 3, 0, 11])
    th = np.pi * (2 * ts + 1) / (2 * N - 1)
    ph = 2 * np.pi * ps / (2 * N - 1)
    ref = np.zeros((len(ts), len(ps)), complex)
    for l in range(N):
        for m in range(-l, l + 1):
            ref += flm[l * l + l + m] * special.sph_harm_y(l, m, th[:, None], ph[None, :])
    assert np.max(np.abs(sht.inverse_at(flm, N, ts, ps) - ref)) < 1e-13

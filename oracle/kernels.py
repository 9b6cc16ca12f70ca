"""ORACLE — test infrastructure only.

Plain FP64 construction of the axisymmetric wavelets and scaling function of
Sect. 2.2, the scale range J, and the band-limits of the multiresolution
algorithm of Sect. 3.1, for two generating-function families:
  "sd"       the smooth scale-discretised generating functions (McEwen et al.
             2008); integrals use scipy's adaptive quadrature (a library
             primitive)
  "bspline"  the cubic B-spline generating function of the footnote of
             Sect. 2.2, k(t) = 3/2 B_3(2 t lambda^(J-1) / L)
Nothing here is shared with the GPU library.
"""
import functools
import math

import numpy as np
from scipy import integrate


def s(t):
    """Bump function s(t) = exp(-1/(1-t^2)) on (-1, 1), zero elsewhere (Sect. 2.2)."""
    if -1.0 < t < 1.0:
        return math.exp(-1.0 / (1.0 - t * t))
    return 0.0


def s_lambda(t, lam):
    """s_lambda(t) = s(2 lambda/(lambda-1) (t - 1/lambda) - 1), support [1/lambda, 1] (Sect. 2.2)."""
    return s(2.0 * lam / (lam - 1.0) * (t - 1.0 / lam) - 1.0)


def _integrand(u, lam):
    return s_lambda(u, lam) ** 2 / u


def _integral(lo, hi, lam):
    val, _ = integrate.quad(_integrand, lo, hi, args=(lam,), epsabs=0.0,
                            epsrel=1e-13, limit=400)
    return val


@functools.lru_cache(maxsize=None)
def _denominator(lam):
    return _integral(1.0 / lam, 1.0, lam)


@functools.lru_cache(maxsize=None)
def k_lambda(t, lam):
    """Eq. (smoothscaling): ratio of the integrals of s_lambda^2(t')/t' over
    [t, 1] and [1/lambda, 1]; unity for t <= 1/lambda, zero for t >= 1."""
    lam = float(lam)
    if t <= 1.0 / lam:
        return 1.0
    if t >= 1.0:
        return 0.0
    return _integral(t, 1.0, lam) / _denominator(lam)


def kappa_lambda(t, lam):
    """Wavelet generating function kappa_lambda(t) = sqrt(k(t/lambda) - k(t)) (Sect. 2.2).

    By Eq. (smoothscaling) the difference of the two ratios is the integral of
    s_lambda^2(t')/t' over [t/lambda, t] (clipped to the support [1/lambda, 1])
    divided by the same denominator; it is evaluated in that form, so that no
    cancellation occurs where both k values are close to 1."""
    lam = float(lam)
    lo = max(t / lam, 1.0 / lam)
    hi = min(t, 1.0)
    if hi <= lo:
        return 0.0
    return math.sqrt(_integral(lo, hi, lam) / _denominator(lam))


def eta_lambda(t, lam):
    """Scaling generating function eta_lambda(t) = sqrt(k(t)) (Sect. 2.2)."""
    return math.sqrt(k_lambda(t, lam))


def jmax(L, B):
    """J = ceil(log_B(L-1)) (Sect. 2.2), evaluated in integers as the smallest
    J >= 0 with B^J >= L-1."""
    J = 0
    while B ** J < L - 1:
        J += 1
    return J


def check_params(L, B, J0):
    J = jmax(L, B)
    if not (L >= 2 and B >= 2 and 0 <= J0 < J):
        raise ValueError("need L >= 2, B >= 2 and 0 <= J0 < J (got L=%d B=%d J0=%d J=%d)"
                         % (L, B, J0, J))
    return J


def psi_l0(L, B, j):
    """Psi^j_l0 = sqrt((2l+1)/(4 pi)) kappa_lambda(l / lambda^j), l < L (Sect. 2.2)."""
    return np.array([math.sqrt((2 * l + 1) / (4 * math.pi)) * kappa_lambda(l / B ** j, B)
                     for l in range(L)])


def phi_l0(L, B, J0):
    """Phi_l0 = sqrt((2l+1)/(4 pi)) eta_lambda(l / lambda^J0), l < L (Sect. 2.2)."""
    return np.array([math.sqrt((2 * l + 1) / (4 * math.pi)) * eta_lambda(l / B ** J0, B)
                     for l in range(L)])


def bandlimits(L, B, J0, multires):
    """Band-limits of the scaling map and of wavelet scales j = J0..J.

    Multiresolution (Sect. 3.1): scale j lives at band-limit min(L, lambda^{j+1});
    the scaling map at min(L, lambda^J0), because eta(l/lambda^J0) = 0 for
    l >= lambda^J0.  Full resolution: every map at L.
    """
    J = check_params(L, B, J0)
    if not multires:
        return L, [L] * (J - J0 + 1)
    return min(L, B ** J0), [min(L, B ** (j + 1)) for j in range(J0, J + 1)]


# ---------------------------------------------------------------- B-spline family
KERNELS = ("sd", "bspline")


def bspline3(x):
    """Cubic B-spline of the footnote of Sect. 2.2, written as its five-term
    sum of cubed distances: (|x-2|^3 - 4|x-1|^3 + 6|x|^3 - 4|x+1|^3 + |x+2|^3) / 12.
    For |x| >= 2 the five cubes cancel identically (the spline's support is
    (-2, 2)); there the exact zero is returned instead of the rounding residue of
    the sum, which grows like |x|^3."""
    if abs(x) >= 2.0:
        return 0.0
    return (abs(x - 2) ** 3 - 4 * abs(x - 1) ** 3 + 6 * abs(x) ** 3 - 4 * abs(x + 1) ** 3
            + abs(x + 2) ** 3) / 12.0


def k_bspline(t, lam, L, J):
    """B-spline generating function k(t) = 3/2 B_3(2 t lambda^(J-1) / L) (footnote of
    Sect. 2.2): 1 at t = 0, decreasing to 0 at t = L / lambda^(J-1)."""
    return 1.5 * bspline3(2.0 * t * float(lam) ** (J - 1) / L)


def psi_l0_bspline(L, B, j, J):
    """Psi^j_l0 = sqrt((2l+1)/(4 pi)) kappa(l / lambda^j) with kappa(t) =
    sqrt(k(t/lambda) - k(t)) (Sect. 2.2) for j < J.  The finest scale j = J
    takes the remainder, kappa_J(l)^2 = 1 - k(l / lambda^J), so that the
    squared kernels of all scales sum to one for every l < L (the reading taken
    here: the paper's telescoping sum would end at k(l / lambda^(J+1)), which
    is 1 only at l = 0 for this k)."""
    out = np.zeros(L)
    for l in range(L):
        if j < J:
            d = k_bspline(l / B ** (j + 1), B, L, J) - k_bspline(l / B ** j, B, L, J)
        else:
            d = 1.0 - k_bspline(l / B ** J, B, L, J)
        out[l] = math.sqrt((2 * l + 1) / (4 * math.pi)) * math.sqrt(max(d, 0.0))
    return out


def phi_l0_bspline(L, B, J0, J):
    """Phi_l0 = sqrt((2l+1)/(4 pi)) sqrt(k(l / lambda^J0)) (Sect. 2.2)."""
    return np.array([math.sqrt((2 * l + 1) / (4 * math.pi)) * math.sqrt(max(k_bspline(l / B ** J0, B, L, J), 0.0))
                     for l in range(L)])


def bandlimits_bspline(L, B, J0, multires):
    """Multiresolution band-limits of the B-spline family (Sect. 3.1): scale j
    lives at min(L, ceil(L / lambda^(J-j-2))), the support of its kernel; the
    scaling map at min(L, ceil(L / lambda^(J-J0-1))), where k(l / lambda^J0)
    vanishes.  Full resolution: every map at L."""
    J = check_params(L, B, J0)
    if not multires:
        return L, [L] * (J - J0 + 1)

    def cap(e):                      # min(L, ceil(L / B^e)), e may be negative
        if e <= 0:
            return L
        d = B ** e
        return min(L, (L + d - 1) // d)

    return cap(J - J0 - 1), [cap(J - j - 2) for j in range(J0, J + 1)]

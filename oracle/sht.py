"""ORACLE — test infrastructure only.

Plain FP64 spherical harmonic transforms on McEwen-Wiaux (MW) equiangular
samples (the sampling theorem adopted in Sect. 2.1).  A map at band-limit N
has N rings theta_t = pi (2t+1)/(2N-1), t = 0..N-1 (t = N-1 is the south
pole), and 2N-1 longitudes phi_p = 2 pi p/(2N-1); it is stored as an
N x (2N-1) array with the pole ring held in full.  Harmonic coefficients are
complex, index l*l + l + m, length N*N, for real and complex maps alike.

  inverse: Eq. (harmonicssynthesis) truncated at l < N, evaluated on the grid.
  forward: Eq. (harmonicsanalysis) as the exact MW quadrature, written out as
           (1) ring DFT, (2) extension of each F_m(theta) to the full circle
           with parity (-1)^m, (3) Fourier coefficients in theta,
           (4) product with the weights w(p) = int_0^pi e^{i p t} sin t dt,
           (5) back to the circle, (6) fold onto the N rings, (7) Legendre sum.
           Exact for band-limited maps because every function of theta that
           appears is a trigonometric polynomial of degree <= N-1.
  *_adjoint: conjugate transposes of the two transforms, step by step in
           reverse order (the transpose under the Euclidean inner product of
           the stored arrays).

Every DFT is written as a product with its explicit e^{...} matrix (numpy
matmul, a library primitive); the Legendre sums call the oracle's own C code.
The GPU library shares none of this.
"""
import decimal
import functools
import math

import numpy as np

from . import _clib


def n_phi(N):
    return 2 * N - 1


def thetas(N, nt=None):
    """MW colatitudes theta_t = pi (2t+1)/(2N-1) for t < nt (default nt = N)."""
    nt = N if nt is None else nt
    return math.pi * (2.0 * np.arange(nt) + 1.0) / (2 * N - 1)


def phis(N):
    return 2.0 * math.pi * np.arange(2 * N - 1) / (2 * N - 1)


_PI_DIGITS = "3.14159265358979323846264338327950288419716939937510582097494459230781640629"


@functools.lru_cache(maxsize=None)
def _sin_cos_pi_ratio(k, P):
    """For theta = pi k / P, 0 <= k <= P: (sin theta, sgn, y) with
    cos theta = sgn (1 - y), sgn = +-1 and y = 1 - |cos theta| >= 0, each
    rounded once from about 45 significant digits (Taylor series in decimal
    arithmetic)."""
    with decimal.localcontext() as ctx:
        ctx.prec = 60
        x = decimal.Decimal(_PI_DIGITS) * k / P
        x2 = x * x
        term_c = decimal.Decimal(1)
        term_s = x
        c = term_c
        s = term_s
        n = 0
        tiny = decimal.Decimal(10) ** -58
        while abs(term_c) > tiny or abs(term_s) > tiny:
            n += 1
            term_c = -term_c * x2 / ((2 * n - 1) * (2 * n))
            term_s = -term_s * x2 / ((2 * n) * (2 * n + 1))
            c += term_c
            s += term_s
        sgn = 1.0 if c >= 0 else -1.0
        y = 1 - abs(c)
        if k == P:  # south pole: sin = 0, cos = -1 exactly
            return 0.0, -1.0, 0.0
        return float(s), sgn, float(y)


def sin_cos_theta(N, ts):
    """(sin theta_t, sgn_t, y_t) with cos theta_t = sgn_t (1 - y_t),
    theta_t = pi (2t+1)/(2N-1).  The south pole (t = N-1) is exact."""
    P = 2 * N - 1
    vals = [_sin_cos_pi_ratio(int(2 * t + 1), P) for t in np.asarray(ts)]
    s = np.array([v[0] for v in vals], dtype=np.float64)
    sg = np.array([v[1] for v in vals], dtype=np.float64)
    y = np.array([v[2] for v in vals], dtype=np.float64)
    return s, sg, y


def weights(p):
    """w(p) = int_0^pi e^{i p theta} sin(theta) dtheta in closed form:
    2/(1-p^2) for even p, +-i pi/2 for p = +-1, 0 for other odd p."""
    p = np.asarray(p)
    out = np.zeros(p.shape, dtype=complex)
    ev = (p % 2) == 0
    out[ev] = 2.0 / (1.0 - p[ev].astype(float) ** 2)
    out[p == 1] = 0.5j * math.pi
    out[p == -1] = -0.5j * math.pi
    return out


def m_range(N):
    return np.arange(-(N - 1), N)


def expi_pi(k, P):
    """exp(i pi k / P) for integer k, with k reduced modulo 2P in integers
    first, so that large k lose no accuracy to argument rounding."""
    k = np.mod(np.asarray(k, dtype=np.int64), 2 * P)
    return np.exp(1j * math.pi * k / P)


def _phase_m_phi(m, p, P):
    """e^{i m phi_p} with phi_p = 2 pi p / P."""
    return expi_pi(2 * np.multiply.outer(np.asarray(m, dtype=np.int64), np.asarray(p, dtype=np.int64)), P)


def _phase_a_theta(a, t, P):
    """e^{i a theta_t} with theta_t = pi (2t+1) / P."""
    return expi_pi(np.multiply.outer(np.asarray(a, dtype=np.int64), 2 * np.asarray(t, dtype=np.int64) + 1), P)


# The constant matrices of one band-limit are built once per process.
@functools.lru_cache(maxsize=8)
def _phase_matrix_phi(N):
    """e^{i m phi_p}, [m + N - 1, p]."""
    return _phase_m_phi(m_range(N), np.arange(2 * N - 1), 2 * N - 1)


@functools.lru_cache(maxsize=8)
def _quadrature_matrices(N):
    """e^{-i a theta_t} [t, a], w(a+b) [a, b] and e^{-i b theta_t} [b, t] on the full circle."""
    P = 2 * N - 1
    a = m_range(N)
    E3 = np.ascontiguousarray(np.conj(_phase_a_theta(a, np.arange(P), P)).T)
    W = weights(a[:, None] + a[None, :])
    E5 = np.conj(_phase_a_theta(a, np.arange(P), P))
    return E3, W, E5


def legendre_column(m, N, sin_t, sgn, y):
    """lambda_lm(theta) for l = m..N-1 (m >= 0); cos(theta) = sgn (1 - y)."""
    out = np.zeros(N - m)
    _clib.lib().oracle_legendre_column(m, N, float(sin_t), float(sgn), float(y),
                                       _clib.dptr(out), None, None)
    return out


def legendre_column_x(m, N, sin_t, sgn, y):
    """lambda_lm(theta), l = m..N-1, as (FP64 value, mantissa, base-2 exponent)."""
    out = np.zeros(N - m)
    f = np.zeros(N - m)
    e = np.zeros(N - m, dtype=np.int32)
    _clib.lib().oracle_legendre_column(m, N, float(sin_t), float(sgn), float(y),
                                       _clib.dptr(out), _clib.dptr(f), _clib.iptr(e))
    return out, f, e


def legendre_at(m, N, t):
    """lambda_lm(theta_t), l = m..N-1, on MW ring t of band-limit N."""
    s, sg, y = sin_cos_theta(N, [t])
    return legendre_column(m, N, s[0], sg[0], y[0])


def _orders(N, orders):
    m = m_range(N) if orders is None else np.asarray(orders, dtype=np.int64)
    return m[np.abs(m) <= N - 1]


def _legendre_inverse(flm, N, ts, orders=None):
    """F_m(theta_t) = sum_l f_lm lambda_lm(theta_t), shape [len(orders), len(ts)]."""
    m = _orders(N, orders)
    s, sg, yy = sin_cos_theta(N, ts)
    fl = np.ascontiguousarray(np.asarray(flm, dtype=complex)[:N * N]).view(np.float64)
    out = np.zeros((len(m), len(ts)), dtype=complex)
    mi = np.ascontiguousarray(m, dtype=np.int32)
    _clib.lib().oracle_legendre_inverse(N, _clib.dptr(fl), len(ts), _clib.dptr(s),
                                        _clib.dptr(sg), _clib.dptr(yy), len(mi), _clib.iptr(mi),
                                        _clib.dptr(out.view(np.float64)))
    return out


def _legendre_forward(G, N, orders=None):
    """out_lm = sum_t lambda_lm(theta_t) G_m(theta_t); G has shape [len(orders), N (t)].
    Coefficients of orders not listed are 0."""
    m = _orders(N, orders)
    s, sg, yy = sin_cos_theta(N, np.arange(N))
    G = np.ascontiguousarray(G, dtype=complex)
    out = np.zeros(N * N, dtype=complex)
    mi = np.ascontiguousarray(m, dtype=np.int32)
    _clib.lib().oracle_legendre_forward(N, _clib.dptr(G.view(np.float64)), N, _clib.dptr(s),
                                        _clib.dptr(sg), _clib.dptr(yy), len(mi), _clib.iptr(mi),
                                        _clib.dptr(out.view(np.float64)))
    return out


def inverse(flm, N, real=False, orders=None):
    """Eq. (harmonicssynthesis): f(theta_t, phi_p) = sum_{l<N} sum_{|m|<=l} f_lm Y_lm.
    With `orders`, only the terms of those orders m are summed."""
    m = _orders(N, orders)
    F = _legendre_inverse(flm, N, np.arange(N), m)       # [m, t]
    E = _phase_matrix_phi(N)[m + N - 1]                   # e^{i m phi_p}, [m, p]
    f = F.T @ E                                           # [t, p]
    return f.real.copy() if real else f


def inverse_at(flm, N, ts, ps):
    """The inverse transform evaluated only at rings ts and longitudes ps."""
    m = m_range(N)
    F = _legendre_inverse(flm, N, np.asarray(ts))
    E = _phase_matrix_phi(N)[:, np.asarray(ps)]
    return F.T @ E


def _theta_quadrature(Fm, N, par):
    """Steps (2)-(6) of the forward transform: from F_m(theta_t), t < N, to the
    folded G_m(theta_t), t < N.  Fm: [rows, N]; par: [rows, 1] holds (-1)^m."""
    P = 2 * N - 1
    # (2) extension to the full circle: F~_m(theta_{P-1-t}) = (-1)^m F_m(theta_t), t <= N-2
    Ft = np.zeros((Fm.shape[0], P), dtype=complex)
    Ft[:, :N] = Fm
    if N > 1:
        Ft[:, N:] = par * Fm[:, N - 2::-1]
    E3, W, E5 = _quadrature_matrices(N)
    # (3) F_{m,a} = (1/P) sum_{t<P} F~_m(theta_t) e^{-i a theta_t},  |a| <= N-1
    Fma = Ft @ E3 / P                                     # [m, a]
    # (4) H_{m,b} = sum_a F_{m,a} w(a+b)
    H = Fma @ W                                           # [m, b]
    # (5) h_m(theta_t) = sum_b H_{m,b} e^{-i b theta_t},  t < P
    h = H @ E5                                            # [m, t]
    # (6) fold: G_m(theta_t) = h_m(theta_t) + (-1)^m h_m(theta_{P-1-t}) for t < N-1
    G = h[:, :N].copy()
    if N > 1:
        G[:, :N - 1] += par * h[:, P - 1 - np.arange(N - 1)]
    return G


def _parity(m):
    return np.where(np.asarray(m) % 2 == 0, 1.0, -1.0).reshape(-1, 1)


def forward(f, N, orders=None):
    """Eq. (harmonicsanalysis) by the exact MW quadrature; returns f_lm, l < N.
    With `orders`, only coefficients of those orders m are computed (others 0):
    every step below acts on each order separately."""
    P = 2 * N - 1
    f = np.asarray(f)
    assert f.shape == (N, P)
    m = _orders(N, orders)
    # (1) F_m(theta_t) = (1/P) sum_p f(theta_t, phi_p) e^{-i m phi_p}
    Fm = (f @ np.conj(_phase_matrix_phi(N)[m + N - 1]).T / P).T  # [m, t]
    G = _theta_quadrature(Fm, N, _parity(m))
    # (7) f_lm = (2 pi / P) sum_{t<N} lambda_lm(theta_t) G_m(theta_t)
    return (2.0 * math.pi / P) * _legendre_forward(G, N, m)


def forward_m(f, N, m):
    """f_lm for one order m and l = |m|..N-1, by the same steps as forward()."""
    P = 2 * N - 1
    f = np.asarray(f)
    Fm = (f @ np.conj(_phase_m_phi([m], np.arange(P), P))[0] / P)[None, :]  # (1), this m only
    G = _theta_quadrature(Fm, N, _parity([m]))[0]         # (2)-(6)
    s, sg, yy = sin_cos_theta(N, np.arange(N))
    am = abs(m)
    sgn = (-1.0) ** am if m < 0 else 1.0                  # lambda_{l,-m} = (-1)^m lambda_lm
    out = np.zeros(N - am, dtype=complex)
    for t in range(N):                                    # (7)
        out += sgn * legendre_column(am, N, s[t], sg[t], yy[t]) * G[t]
    return (2.0 * math.pi / P) * out


# ---------------------------------------------------------------- adjoints
def inverse_adjoint(g, N):
    """Conjugate transpose of inverse(): out_lm = sum_{t,p} g(theta_t, phi_p)
    lambda_lm(theta_t) e^{-i m phi_p}."""
    m = m_range(N)
    g = np.asarray(g, dtype=complex)
    Gm = (g @ np.conj(_phase_matrix_phi(N)).T).T          # [m, t]
    return _legendre_forward(Gm, N)


def forward_adjoint(y, N):
    """Conjugate transpose of forward(), each step of forward() transposed in
    reverse order."""
    P = 2 * N - 1
    m = m_range(N)
    par = np.where(m % 2 == 0, 1.0, -1.0)[:, None]
    # (7)^H: G_m(theta_t) = (2 pi / P) sum_l lambda_lm(theta_t) y_lm
    G = (2.0 * math.pi / P) * _legendre_inverse(y, N, np.arange(N))   # [m, t]
    # (6)^H: h(theta_t) = G(theta_t) for t < N; h(theta_{P-1-t}) = (-1)^m G(theta_t) for t < N-1
    h = np.zeros((len(m), P), dtype=complex)
    h[:, :N] = G
    if N > 1:
        h[:, P - 1 - np.arange(N - 1)] = par * G[:, :N - 1]
    a = m_range(N)
    # (5)^H
    H = h @ _phase_a_theta(a, np.arange(P), P).T          # [m, b]
    # (4)^H
    Fma = H @ np.conj(weights(a[:, None] + a[None, :])).T  # [m, a]
    # (3)^H
    Ft = Fma @ _phase_a_theta(a, np.arange(P), P) / P     # [m, t]
    # (2)^H
    Fm = Ft[:, :N].copy()
    if N > 1:
        Fm[:, :N - 1] += par * Ft[:, P - 1 - np.arange(N - 1)]
    # (1)^H: f(theta_t, phi_p) = (1/P) sum_m F_m(theta_t) e^{i m phi_p}
    return Fm.T @ _phase_m_phi(m, np.arange(P), P) / P

"""Seeded synthetic inputs: random harmonic coefficients.

This module only draws random numbers; it holds none of the transform's
arithmetic, so both the GPU path and the CPU oracle can take their inputs
from it.  Coefficients are complex, index l*l + l + m, l < L.

Workload recipe (the paper's validation draws f_lm from independent Gaussians,
Sect. 3.3):
  spectrum "white": E|f_lm|^2 = 1 for every l.
  spectrum "cl":    E|f_lm|^2 = C_l = 1/(l(l+1)) for l >= 2, C_0 = C_1 = 0.
  real=True:  f_l0 real N(0, C_l); for m > 0 real and imaginary parts are
              N(0, C_l/2); f_{l,-m} = (-1)^m conj(f_lm) so the map is real.
  real=False: every (l, m) independent, real and imaginary parts N(0, C_l/2).
"""
import numpy as np


def spectrum(L, kind):
    l = np.arange(L, dtype=np.float64)
    if kind == "white":
        return np.ones(L)
    if kind == "cl":
        c = np.zeros(L)
        c[2:] = 1.0 / (l[2:] * (l[2:] + 1.0))
        return c
    raise ValueError("unknown spectrum %r" % (kind,))


def random_flm(L, seed, real=True, kind="white"):
    """One set of coefficients, shape (L*L,), complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cl = spectrum(L, kind)
    n = L * L
    zr = rng.standard_normal(n)
    zi = rng.standard_normal(n)
    l = np.repeat(np.arange(L), 2 * np.arange(L) + 1)
    m = np.arange(n) - l * l - l
    amp = np.sqrt(cl[l] / 2.0)
    flm = amp * (zr + 1j * zi)
    if real:
        flm[m == 0] = np.sqrt(cl[l[m == 0]]) * zr[m == 0]
        neg = m < 0
        partner = l[neg] * l[neg] + l[neg] - m[neg]
        flm[neg] = ((-1.0) ** (-m[neg])) * np.conj(flm[partner])
    return flm


def random_flm_batch(L, seeds, real=True, kind="white"):
    """Coefficients for several maps, shape (len(seeds), L*L)."""
    return np.stack([random_flm(L, s, real, kind) for s in seeds])


def random_map(shape, seed, real=True):
    """Independent N(0,1) samples (not band-limited), for adjoint tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal(shape)
    if not real:
        x = x + 1j * rng.standard_normal(shape)
    return x

"""ORACLE — test infrastructure only.

Plain FP64 axisymmetric scale-discretised wavelet transform on MW samples:

  analysis  (Eqs. wav2, wav4; multiresolution of Sect. 3.1):
      f_lm = forward_L(f)
      W^Phi_lm = sqrt(4 pi/(2l+1)) f_lm Phi*_l0,   map at the scaling band-limit
      W^j_lm   = sqrt(4 pi/(2l+1)) f_lm Psi^j*_l0, map at scale j's band-limit
  synthesis (Eq. waveletsynthesis):
      f_lm = sqrt(4 pi/(2l+1)) [W^Phi_lm Phi_l0 + sum_j W^j_lm Psi^j_l0],
      with W_lm = forward_N(W) of each map, then f = inverse_L(f_lm)
  adjoint of the analysis: the conjugate transpose of each step in reverse
      order (for real maps this is the transpose under the Euclidean inner
      product of the stored samples).

Maps are lists of arrays: f_wav[j - J0] has shape (N_j, 2 N_j - 1).
"""
import math

import numpy as np

from . import kernels, sht


def _ell_index(N):
    """l for every index l*l + l + m, l < N."""
    return np.repeat(np.arange(N), 2 * np.arange(N) + 1)


def _norm(N):
    l = _ell_index(N)
    return np.sqrt(4.0 * math.pi / (2.0 * l + 1.0))


def tables(L, B, J0, kernel="sd"):
    """(Phi_l0, [Psi^j_l0 for j = J0..J]) for l < L, of the generating-function
    family `kernel` ("sd" or "bspline")."""
    J = kernels.check_params(L, B, J0)
    if kernel == "bspline":
        return (kernels.phi_l0_bspline(L, B, J0, J),
                [kernels.psi_l0_bspline(L, B, j, J) for j in range(J0, J + 1)])
    if kernel != "sd":
        raise ValueError("kernel must be 'sd' or 'bspline'")
    phi = kernels.phi_l0(L, B, J0)
    psi = [kernels.psi_l0(L, B, j) for j in range(J0, J + 1)]
    return phi, psi


def bandlimits(L, B, J0, multires, kernel="sd"):
    """Band-limits of the scaling map and of scales J0..J for the family."""
    if kernel == "bspline":
        return kernels.bandlimits_bspline(L, B, J0, multires)
    return kernels.bandlimits(L, B, J0, multires)


def _expand(per_l, N):
    return np.asarray(per_l)[_ell_index(N)]


def analysis_lm(flm, L, B, J0, multires=True, kernel="sd"):
    """Harmonic coefficients of the scaling map and wavelet maps, each truncated
    at its band-limit (Eqs. wav2, wav4)."""
    phi, psi = tables(L, B, J0, kernel)
    n_scal, n_wav = bandlimits(L, B, J0, multires, kernel)
    c = _norm(L) * flm[:L * L]
    scal = (c * np.conj(_expand(phi, L)))[:n_scal * n_scal]
    wav = [(c * np.conj(_expand(p, L)))[:n * n] for p, n in zip(psi, n_wav)]
    return scal, wav


def analysis(f, L, B, J0, multires=True, real=True, orders=None, kernel="sd"):
    """With `orders`, only the parts of those orders m are computed: every step
    acts on each order separately, so the result is the order-m component of
    the full analysis (used to time a bounded sample of one map)."""
    flm = sht.forward(f, L, orders)
    scal_lm, wav_lm = analysis_lm(flm, L, B, J0, multires, kernel)
    n_scal, n_wav = bandlimits(L, B, J0, multires, kernel)
    f_scal = sht.inverse(scal_lm, n_scal, real=real, orders=orders)
    f_wav = [sht.inverse(w, n, real=real, orders=orders) for w, n in zip(wav_lm, n_wav)]
    return f_wav, f_scal


def _pad(xlm, L):
    out = np.zeros(L * L, dtype=complex)
    out[:len(xlm)] = xlm
    return out


def synthesis_lm(scal_lm, wav_lm, L, B, J0, kernel="sd"):
    """Eq. (waveletsynthesis) in harmonic space."""
    phi, psi = tables(L, B, J0, kernel)
    c = _norm(L)
    flm = c * _pad(scal_lm, L) * _expand(phi, L)
    for w, p in zip(wav_lm, psi):
        flm = flm + c * _pad(w, L) * _expand(p, L)
    return flm


def synthesis(f_wav, f_scal, L, B, J0, multires=True, real=True, orders=None, kernel="sd"):
    """With `orders`, only the parts of those orders m (see analysis())."""
    n_scal, n_wav = bandlimits(L, B, J0, multires, kernel)
    scal_lm = sht.forward(f_scal, n_scal, orders)
    wav_lm = [sht.forward(w, n, orders) for w, n in zip(f_wav, n_wav)]
    flm = synthesis_lm(scal_lm, wav_lm, L, B, J0, kernel)
    return sht.inverse(flm, L, real=real, orders=orders)


def analysis_adjoint(g_wav, g_scal, L, B, J0, multires=True, real=True, kernel="sd"):
    """Conjugate transpose of analysis(): sum over maps of
    forward_L^H diag(conj(c)) inverse_N^H, with c the kernel factor of each map."""
    phi, psi = tables(L, B, J0, kernel)
    n_scal, n_wav = bandlimits(L, B, J0, multires, kernel)
    c = _norm(L)
    ylm = np.conj(c * np.conj(_expand(phi, L))) * _pad(sht.inverse_adjoint(g_scal, n_scal), L)
    for g, p, n in zip(g_wav, psi, n_wav):
        ylm = ylm + np.conj(c * np.conj(_expand(p, L))) * _pad(sht.inverse_adjoint(g, n), L)
    out = sht.forward_adjoint(ylm, L)
    return out.real.copy() if real else out


# ---------------------------------------------------------------- denoising (Sect. 4.3)
def noise_std(L, B, J0, kernel="sd"):
    """(sigma^Phi / sigma, [sigma^j / sigma for j = J0..J]): the standard deviation,
    per unit harmonic noise variance, of white noise in the scaling map and in
    wavelet scale j, sqrt(sum_l |Psi^j_l0|^2) (Eq. noisemodel)."""
    phi, psi = tables(L, B, J0, kernel)
    return math.sqrt(float(np.sum(phi ** 2))), [math.sqrt(float(np.sum(p ** 2))) for p in psi]


def hard_threshold(f_wav, sigma, L, B, J0, nsigma=3.0, kernel="sd"):
    """Eq. (threshold) with T^j = nsigma sigma^j: a sample of scale j is set to zero
    where its modulus is below T^j and kept otherwise (the paper writes the test
    on the signed coefficient; the modulus is the reading taken here)."""
    _, s_j = noise_std(L, B, J0, kernel)
    return [np.where(np.abs(w) < nsigma * sigma * s, 0.0 * w, w) for w, s in zip(f_wav, s_j)]


def denoise(y, sigma, L, B, J0, multires=True, real=True, nsigma=3.0, kernel="sd"):
    """Sect. 4.3: wavelet analysis of the noisy map, hard thresholding of the wavelet
    maps (the scaling map is kept), synthesis."""
    f_wav, f_scal = analysis(y, L, B, J0, multires, real, kernel=kernel)
    d_wav = hard_threshold(f_wav, sigma, L, B, J0, nsigma, kernel)
    return synthesis(d_wav, f_scal, L, B, J0, multires, real, kernel=kernel)


def snr_db(s, y, L):
    """SNR(y) = 10 log10(||s||^2 / ||y - s||^2) with ||.||^2 the sum of |f_lm|^2 (Sect. 4.3)."""
    ds = sht.forward(s, L)
    dn = sht.forward(y - s, L)
    return 10.0 * math.log10(float(np.sum(np.abs(ds) ** 2)) / float(np.sum(np.abs(dn) ** 2)))

"""Pins for the oracle's wavelet analysis, synthesis and analysis-adjoint
(Eqs. wav2, wav4, waveletsynthesis; multiresolution of Sect. 3.1)."""
import math

import numpy as np
import pytest

from oracle import kernels, sht, wavelet
from paper_1211_1680_gb300 import inputs

CASES = [  # (L, B, J0, multires, real)
    (32, 2, 0, False, True),    # the L=32 full-resolution workload
    (32, 2, 0, True, True),
    (40, 3, 1, True, False),
    (27, 3, 2, False, False),
    (64, 2, 2, True, True),
]


@pytest.mark.parametrize("L,B,J0,multires,real", CASES)
def test_exact_reconstruction(L, B, J0, multires, real):
    """Synthesis after analysis returns the band-limited map (Eq. identity)."""
    f = sht.inverse(inputs.random_flm(L, 7, real=real), L, real=real)
    fw, fs = wavelet.analysis(f, L, B, J0, multires, real)
    n_scal, n_wav = kernels.bandlimits(L, B, J0, multires)
    assert fs.shape == (n_scal, 2 * n_scal - 1)
    assert [w.shape for w in fw] == [(n, 2 * n - 1) for n in n_wav]
    fr = wavelet.synthesis(fw, fs, L, B, J0, multires, real)
    assert np.max(np.abs(fr - f)) / np.max(np.abs(f)) < 1e-13


@pytest.mark.parametrize("ell", [0, 3, 7, 12, 20])
def test_axisymmetric_input(ell):
    """f = Y_l0: Eq. (wav2) gives W^j = sqrt(4 pi/(2l+1)) Psi^j_l0 Y_l0, i.e.
    kappa(l/lambda^j) Y_l0, at every scale's band-limit."""
    L, B, J0 = 24, 2, 1
    flm = np.zeros(L * L, complex)
    flm[ell * ell + ell] = 1.0
    f = sht.inverse(flm, L, real=True)
    fw, fs = wavelet.analysis(f, L, B, J0, True, True)
    n_scal, n_wav = kernels.bandlimits(L, B, J0, True)
    for j, (w, n) in enumerate(zip(fw, n_wav), start=J0):
        ref = np.zeros(n * n, complex)
        if ell < n:
            ref[ell * ell + ell] = kernels.kappa_lambda(ell / B ** j, B)
        assert np.max(np.abs(w - sht.inverse(ref, n, real=True))) < 1e-13
    ref = np.zeros(n_scal * n_scal, complex)
    if ell < n_scal:
        ref[ell * ell + ell] = kernels.eta_lambda(ell / B ** J0, B)
    assert np.max(np.abs(fs - sht.inverse(ref, n_scal, real=True))) < 1e-13


def test_multires_matches_full_resolution():
    """Sect. 3.1: the multiresolution maps hold the same information as the
    full-resolution ones: their harmonic coefficients agree and the
    full-resolution maps have none above the scale band-limit."""
    L, B, J0 = 48, 2, 1
    f = sht.inverse(inputs.random_flm(L, 11, real=True), L, real=True)
    fw_m, fs_m = wavelet.analysis(f, L, B, J0, True, True)
    fw_f, fs_f = wavelet.analysis(f, L, B, J0, False, True)
    n_scal, n_wav = kernels.bandlimits(L, B, J0, True)
    pairs = list(zip(fw_m, fw_f, n_wav)) + [(fs_m, fs_f, n_scal)]
    for wm, wf, n in pairs:
        lm_m = sht.forward(wm, n)
        lm_f = sht.forward(wf, L)
        assert np.max(np.abs(lm_f[:n * n] - lm_m)) < 1e-13
        assert np.max(np.abs(lm_f[n * n:])) < 1e-13 if n < L else True


@pytest.mark.parametrize("L,B,J0,multires,real", CASES[1:] + [(16, 2, 1, False, True)])
def test_adjoint_dot_product(L, B, J0, multires, real):
    """<A x, y> = <x, A^T y> on random (not band-limited) arrays."""
    x = inputs.random_map((L, 2 * L - 1), 31, real=real)
    fw, fs = wavelet.analysis(x, L, B, J0, multires, real)
    gw = [inputs.random_map(w.shape, 40 + i, real=real) for i, w in enumerate(fw)]
    gs = inputs.random_map(fs.shape, 39, real=real)
    lhs = sum(np.vdot(g, w) for g, w in zip(gw, fw)) + np.vdot(gs, fs)
    rhs = np.vdot(wavelet.analysis_adjoint(gw, gs, L, B, J0, multires, real), x)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_dense_transpose():
    """At L = 4 build the analysis matrix and the adjoint matrix column by
    column; the second is the transpose of the first."""
    L, B, J0 = 4, 2, 0
    for multires in (True, False):
        n_in = L * (2 * L - 1)
        cols = []
        for k in range(n_in):
            e = np.zeros(n_in)
            e[k] = 1.0
            fw, fs = wavelet.analysis(e.reshape(L, 2 * L - 1), L, B, J0, multires, True)
            cols.append(np.concatenate([fs.ravel()] + [w.ravel() for w in fw]))
        A = np.array(cols).T
        shapes = [fs.shape] + [w.shape for w in fw]
        sizes = [a * b for a, b in shapes]
        rows = []
        for k in range(A.shape[0]):
            e = np.zeros(A.shape[0])
            e[k] = 1.0
            parts = np.split(e, np.cumsum(sizes)[:-1])
            gs = parts[0].reshape(shapes[0])
            gw = [p.reshape(s) for p, s in zip(parts[1:], shapes[1:])]
            rows.append(wavelet.analysis_adjoint(gw, gs, L, B, J0, multires, True).ravel())
        At = np.array(rows).T
        assert np.max(np.abs(At - A.T)) < 1e-14


def test_white_noise_variance():
    """Wavelet-space noise (Sect. 4.3): for white harmonic noise of variance
    sigma^2, E|W^j|^2 = sigma^2 sum_l |Psi^j_l0|^2 at every sample.  Averaged over
    the samples of several realisations it must agree to a few per cent."""
    L, B, J0 = 64, 2, 2
    phi, psi = wavelet.tables(L, B, J0)
    n_scal, n_wav = kernels.bandlimits(L, B, J0, True)
    acc = [0.0] * len(psi)
    reps = 6
    for r in range(reps):
        flm = inputs.random_flm(L, 500 + r, real=False)
        scal_lm, wav_lm = wavelet.analysis_lm(flm, L, B, J0, True)
        for i, (w, n) in enumerate(zip(wav_lm, n_wav)):
            acc[i] += np.mean(np.abs(sht.inverse(w, n)) ** 2) / reps
    for i, p in enumerate(psi):
        if n_wav[i] >= 16:
            assert acc[i] == pytest.approx(np.sum(p ** 2), rel=0.08)


def test_round_trip_by_orders():
    """Analysis and synthesis restricted to a set of orders give exactly the
    order-restricted components of the full transforms."""
    L, B, J0 = 12, 2, 1
    f = sht.inverse(inputs.random_flm(L, 17, real=True), L, real=True)
    fw, fs = wavelet.analysis(f, L, B, J0, True, True)
    allm = list(range(-(L - 1), L))
    fw_o, fs_o = wavelet.analysis(f, L, B, J0, True, False, orders=allm)
    assert np.max(np.abs(fs_o - fs)) < 1e-13
    for a, b in zip(fw_o, fw):
        assert np.max(np.abs(a - b)) < 1e-13
    sub = [-5, 0, 3, 11]
    fw_s, fs_s = wavelet.analysis(f, L, B, J0, True, False, orders=sub)
    rec = wavelet.synthesis(fw_s, fs_s, L, B, J0, True, False, orders=sub)
    flm = sht.forward(f, L)
    keep = np.zeros(L * L, complex)
    for l in range(L):
        for m in sub:
            if abs(m) <= l:
                keep[l * l + l + m] = flm[l * l + l + m]
    assert np.max(np.abs(rec - sht.inverse(keep, L))) < 1e-13
    # the sampled wavelet maps are the order-restricted parts of the full ones
    n_scal, n_wav = kernels.bandlimits(L, B, J0, True)
    for w_s, w, n in zip(fw_s, fw, n_wav):
        ref = sht.inverse(np.where(np.isin(np.arange(n * n) - np.repeat(np.arange(n), 2 * np.arange(n) + 1) ** 2
                                           - np.repeat(np.arange(n), 2 * np.arange(n) + 1), sub),
                                   sht.forward(w, n), 0), n)
        assert np.max(np.abs(w_s - ref)) < 1e-13


@pytest.mark.parametrize("L,B,J0,multires,real", [(32, 2, 0, True, True), (40, 3, 1, True, False),
                                                  (33, 2, 1, False, True)])
def test_bspline_exact_reconstruction(L, B, J0, multires, real):
    """B-spline generating functions (footnote of Sect. 2.2): synthesis after analysis
    returns the map, with every scale at its (wider) multiresolution band-limit."""
    f = sht.inverse(inputs.random_flm(L, 9, real=real), L, real=real)
    fw, fs = wavelet.analysis(f, L, B, J0, multires, real, kernel="bspline")
    n_scal, n_wav = wavelet.bandlimits(L, B, J0, multires, "bspline")
    assert fs.shape == (n_scal, 2 * n_scal - 1)
    assert [w.shape for w in fw] == [(n, 2 * n - 1) for n in n_wav]
    fr = wavelet.synthesis(fw, fs, L, B, J0, multires, real, kernel="bspline")
    assert np.max(np.abs(fr - f)) / np.max(np.abs(f)) < 1e-13


def test_bspline_multires_matches_full_resolution():
    """The B-spline multiresolution maps hold the full-resolution maps' harmonic
    content: the band-limits are the kernels' supports (Sect. 3.1)."""
    L, B, J0 = 48, 2, 1
    f = sht.inverse(inputs.random_flm(L, 13, real=True), L, real=True)
    fw_m, fs_m = wavelet.analysis(f, L, B, J0, True, True, kernel="bspline")
    fw_f, fs_f = wavelet.analysis(f, L, B, J0, False, True, kernel="bspline")
    n_scal, n_wav = wavelet.bandlimits(L, B, J0, True, "bspline")
    for wm, wf, n in list(zip(fw_m, fw_f, n_wav)) + [(fs_m, fs_f, n_scal)]:
        lm_m = sht.forward(wm, n)
        lm_f = sht.forward(wf, L)
        assert np.max(np.abs(lm_f[:n * n] - lm_m)) < 1e-13
        assert np.max(np.abs(lm_f[n * n:])) < 1e-13 if n < L else True


# ---------------------------------------------------------------- denoising (Sect. 4.3)
@pytest.mark.parametrize("L,B,J0,kernel", [(32, 2, 0, "sd"), (64, 3, 1, "sd"), (48, 2, 1, "bspline")])
def test_noise_std_closed_form(L, B, J0, kernel):
    """By admissibility the squared noise ratios of all maps sum to
    sum_l (2l+1)/(4 pi) = L^2/(4 pi)."""
    s_phi, s_j = wavelet.noise_std(L, B, J0, kernel)
    assert s_phi ** 2 + sum(s * s for s in s_j) == pytest.approx(L * L / (4 * math.pi), rel=1e-13)


def test_noise_std_against_simulated_noise():
    """White noise of harmonic variance sigma^2 (Eq. noisevar), passed through the
    wavelet analysis, has per-sample variance (sigma^j)^2 in every scale (Eq.
    noisemodel): checked on the wavelet maps' samples over 40 realisations."""
    L, B, J0, sigma = 16, 2, 0, 0.7
    rng = np.random.default_rng(5)
    s_phi, s_j = wavelet.noise_std(L, B, J0)
    acc = None
    for _ in range(40):
        nlm = sigma * (rng.standard_normal(L * L) + 1j * rng.standard_normal(L * L)) / math.sqrt(2.0)
        n = sht.inverse(nlm, L, real=False)
        fw, fs = wavelet.analysis(n, L, B, J0, False, False)
        ms = [float(np.mean(np.abs(w) ** 2)) for w in fw] + [float(np.mean(np.abs(fs) ** 2))]
        acc = ms if acc is None else [a + b for a, b in zip(acc, ms)]
    got = [a / 40 for a in acc]
    want = [(sigma * s) ** 2 for s in s_j] + [(sigma * s_phi) ** 2]
    for g, w in zip(got, want):
        if w > 1e-6:
            assert g == pytest.approx(w, rel=0.1)


def test_hard_threshold_semantics():
    """Samples with modulus below 3 sigma^j become zero, the others (and the
    threshold itself) are kept; complex samples compare their modulus."""
    L, B, J0, sigma = 16, 2, 1, 0.5
    _, s_j = wavelet.noise_std(L, B, J0)
    T = [3 * sigma * s for s in s_j]
    fw = [np.array([[0.5 * t, -0.5 * t, 1.5 * t, -1.5 * t, t, 0.999999 * t]]) for t in T]
    out = wavelet.hard_threshold(fw, sigma, L, B, J0)
    for o, t in zip(out, T):
        assert o.tolist() == [[0.0, 0.0, 1.5 * t, -1.5 * t, t, 0.0]]
    fc = [np.array([0.8 * t + 0.5j * t, 0.5 * t - 0.5j * t]) for t in T]   # moduli 0.943 t, 0.707 t
    outc = wavelet.hard_threshold(fc, sigma / 0.9, L, B, J0)   # thresholds 3.33 sigma^j: both below
    assert all(np.all(o == 0) for o in outc)
    outc = wavelet.hard_threshold(fc, sigma * 0.9, L, B, J0)   # thresholds 0.9 T: the first is kept
    for o, f in zip(outc, fc):
        assert o[0] == f[0] and o[1] == 0


def spot_signal(L, spots=((0.9, 1.0, 1.0), (2.0, 4.0, -0.8), (1.4, 2.5, 0.6)), width=0.12):
    """A band-limited real map of a few localised Gaussian spots (theta, phi,
    amplitude): the kind of signal whose wavelet coefficients are sparse."""
    th = np.pi * (2 * np.arange(L) + 1) / (2 * L - 1)
    ph = 2 * np.pi * np.arange(2 * L - 1) / (2 * L - 1)
    T, P = np.meshgrid(th, ph, indexing="ij")
    raw = np.zeros_like(T)
    for t0, p0, a in spots:
        c = np.sin(T) * np.sin(t0) * np.cos(P - p0) + np.cos(T) * np.cos(t0)
        raw += a * np.exp(-np.arccos(np.clip(c, -1.0, 1.0)) ** 2 / (2 * width ** 2))
    return sht.inverse(sht.forward(raw, L), L, real=True)


def test_denoising_raises_snr():
    """Localised spots plus white noise of harmonic variance sigma^2 (Eq. noisevar)
    at SNR(y) near 5 dB: hard thresholding at 3 sigma^j (Eq. threshold) removes
    most of the noise and raises the SNR by several dB (Sect. 4.3)."""
    L, B, J0 = 32, 2, 0
    s = spot_signal(L)
    energy = float(np.sum(np.abs(sht.forward(s, L)) ** 2))
    sigma = math.sqrt(energy / (L * L) / 10 ** 0.5)
    y = s + sht.inverse(sigma * inputs.random_flm(L, 8, True, "white"), L, real=True)
    snr_y = wavelet.snr_db(s, y, L)
    assert 4.0 < snr_y < 6.0
    d = wavelet.denoise(y, sigma, L, B, J0, multires=True, real=True)
    assert wavelet.snr_db(s, d, L) > snr_y + 5.0


@pytest.mark.parametrize("L,B,J0,multires,real", [(24, 2, 1, True, True), (20, 3, 0, True, False),
                                                  (16, 2, 0, False, True)])
def test_bspline_adjoint_dot_product(L, B, J0, multires, real):
    """<A x, y> = <x, A^T y> for the B-spline transform, with its own band-limits."""
    x = inputs.random_map((L, 2 * L - 1), 51, real=real)
    fw, fs = wavelet.analysis(x, L, B, J0, multires, real, kernel="bspline")
    gw = [inputs.random_map(w.shape, 60 + i, real=real) for i, w in enumerate(fw)]
    gs = inputs.random_map(fs.shape, 59, real=real)
    lhs = sum(np.vdot(g, w) for g, w in zip(gw, fw)) + np.vdot(gs, fs)
    rhs = np.vdot(wavelet.analysis_adjoint(gw, gs, L, B, J0, multires, real, kernel="bspline"), x)
    assert lhs == pytest.approx(rhs, rel=1e-12)

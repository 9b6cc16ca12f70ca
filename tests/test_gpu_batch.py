"""Uneven batches (maps of different L and B in one graph launch) against the
oracle, map by map; the captured graph is replayed a second time."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kernels, sht, wavelet  # noqa: E402
from paper_1211_1680_gb300 import _lib, inputs  # noqa: E402
from paper_1211_1680_gb300.s2let import BatchPlan  # noqa: E402
from tests.gpu_util import TOL, from_dev_map, rel_err  # noqa: E402


@pytest.mark.parametrize("real,prec", [(False, "fp32"), (True, "fp64"), (False, "tf32x3")])
def test_uneven_batch_round_trip(real, prec):
    Ls = [16, 24, 9, 16, 33, 24, 16]
    Bs = [2, 3, 3, 2, 2, 3, 3]
    J0 = 1
    bp = BatchPlan(Ls, Bs, J0, real=real, multires=True, precision=prec)
    assert bp.n_groups == len(set(zip(Ls, Bs)))
    f, fw, fs, fo = bp.buffers()
    maps = []
    for i, (L, B) in enumerate(zip(Ls, Bs)):
        x = sht.inverse(inputs.random_flm(L, 40 + i, real), L, real=real)
        maps.append(x)
        xv = x if real else np.stack([x.real, x.imag], -1)
        bp.map_view(f, i).copy_(torch.from_numpy(np.ascontiguousarray(xv)))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for rep in range(2):                      # capture, then replay
            fo.fill_(float("nan"))
            bp.round_trip(f, fw, fs, fo)
            stream.synchronize()
            for i, (L, B) in enumerate(zip(Ls, Bs)):
                got = from_dev_map(bp.map_view(fo, i), real)
                assert rel_err(got, maps[i]) < TOL[prec], (rep, i)
    # wavelet maps of every map against the oracle's analysis
    lib = _lib.lib()
    for i, (L, B) in enumerate(zip(Ls, Bs)):
        _, _, g, k = bp.layout[i]
        ph, _, wav_off, _ = bp.groups[g]
        ref_w, ref_s = wavelet.analysis(maps[i], L, B, J0, True, real)
        n_scal, n_wav = kernels.bandlimits(L, B, J0, True)
        for j, ref in zip(range(J0, J0 + len(n_wav)), ref_w):
            n = ctypes.c_int()
            off = ctypes.c_int64()
            cnt = ctypes.c_int64()
            assert lib.s2let_wav_layout(ctypes.c_void_p(ph), j, ctypes.byref(n), ctypes.byref(off),
                                        ctypes.byref(cnt)) == 0
            per = n.value * (2 * n.value - 1) * (1 if real else 2)
            start = wav_off + off.value + k * per
            shape = (n.value, 2 * n.value - 1) if real else (n.value, 2 * n.value - 1, 2)
            got = from_dev_map(fw[start:start + per].view(shape), real)
            assert rel_err(got, ref) < TOL[prec], (i, j)


def test_autotuned_batch_round_trip():
    """s2let_batch_autotune before the first round trip and again between two
    (the cached graph is dropped and captured with the new choices)."""
    Ls = [16, 40, 9, 40]
    Bs = [2, 2, 3, 2]
    real, prec = True, "tf32x3"
    bp = BatchPlan(Ls, Bs, 1, real=real, multires=True, precision=prec)
    f, fw, fs, fo = bp.buffers()
    maps = []
    for i, (L, B) in enumerate(zip(Ls, Bs)):
        x = sht.inverse(inputs.random_flm(L, 70 + i, real), L, real=real)
        maps.append(x)
        bp.map_view(f, i).copy_(torch.from_numpy(np.ascontiguousarray(x)))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bp.autotune()
        for rep in range(3):
            if rep == 2:
                bp.autotune()
            fo.fill_(float("nan"))
            bp.round_trip(f, fw, fs, fo)
            stream.synchronize()
            for i in range(len(Ls)):
                assert rel_err(from_dev_map(bp.map_view(fo, i), real), maps[i]) < TOL[prec], (rep, i)


def _wavelet_view(bp, fw, i, j, real):
    """The scale-j wavelet map of map i inside the batch's flat f_wav buffer."""
    lib = _lib.lib()
    _, _, g, k = bp.layout[i]
    ph, _, wav_off, _ = bp.groups[g]
    n = ctypes.c_int()
    off = ctypes.c_int64()
    cnt = ctypes.c_int64()
    assert lib.s2let_wav_layout(ctypes.c_void_p(ph), j, ctypes.byref(n), ctypes.byref(off), ctypes.byref(cnt)) == 0
    per = n.value * (2 * n.value - 1) * (1 if real else 2)
    start = wav_off + off.value + k * per
    shape = (n.value, 2 * n.value - 1) if real else (n.value, 2 * n.value - 1, 2)
    return n.value, fw[start:start + per].view(shape)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_uneven_complex_batch_with_large_maps(prec):
    """A reduced uneven batch of the batching workload (complex maps, B in {2, 3},
    J_min = 1) that includes L = 1024 and 512: every map's wavelet maps of every
    scale on sampled rings against the oracle's direct sum of Eq. wav2 from its
    coefficients, and every map's reconstruction against its input."""
    Ls = [1024, 128, 512, 128, 256]
    Bs = [2, 3, 3, 2, 2]
    J0, real = 1, False
    bp = BatchPlan(Ls, Bs, J0, real=real, multires=True, precision=prec)
    f, fw, fs, fo = bp.buffers()
    flms, maps = [], []
    for i, L in enumerate(Ls):
        flm = inputs.random_flm(L, 4000 + i, real)
        x = sht.inverse(flm, L)
        flms.append(flm)
        maps.append(x)
        bp.map_view(f, i).copy_(torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], -1))))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bp.round_trip(f, fw, fs, fo)
        stream.synchronize()
    for i, (L, B) in enumerate(zip(Ls, Bs)):
        assert rel_err(from_dev_map(bp.map_view(fo, i), real), maps[i]) < TOL[prec], ("round trip", i)
        _, psi = wavelet.tables(L, B, J0)
        l_of = np.repeat(np.arange(L), 2 * np.arange(L) + 1)
        norm = np.sqrt(4 * np.pi / (2 * l_of + 1))
        for j, kern in zip(range(J0, J0 + len(psi)), psi):
            n, view = _wavelet_view(bp, fw, i, j, real)
            rings = sorted({0, 1, n // 3, n // 2, n - 2, n - 1} & set(range(n)))
            ref = sht.inverse_at((norm * flms[i] * kern[l_of])[:n * n], n, rings, np.arange(2 * n - 1))
            got = from_dev_map(view, real)[rings]
            assert np.max(np.abs(got - ref)) / np.max(np.abs(from_dev_map(view, real))) < TOL[prec], (i, j)

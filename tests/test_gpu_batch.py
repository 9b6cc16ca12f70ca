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

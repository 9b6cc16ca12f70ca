"""CPU checks of the library's host-side tables through its host-only C-ABI
queries (no GPU): the band-limits and the kernel factors that every plan
uses, against the oracle (Sects. 2.2 and 3.1, footnote of Sect. 2.2)."""
import ctypes
import math

import numpy as np
import pytest

from oracle import kernels, wavelet
from paper_1211_1680_gb300 import _lib

FLAGS = {"sd": 0, "bspline": _lib.S2LET_KERNEL_BSPLINE}


@pytest.mark.parametrize("kernel", ["sd", "bspline"])
@pytest.mark.parametrize("multires", [True, False])
@pytest.mark.parametrize("L,B,J0", [(2048, 2, 2), (1024, 2, 0), (130, 3, 1), (500, 3, 0), (3, 2, 0), (65, 2, 5),
                                    (2000, 5, 1)])
def test_bandlimits_match_oracle(L, B, J0, multires, kernel):
    lib = _lib.lib()
    flags = FLAGS[kernel] | (_lib.S2LET_MULTIRES if multires else 0)
    n_scal = ctypes.c_int()
    nw = (ctypes.c_int * 64)()
    ns = lib.s2let_wav_bandlimits(L, B, J0, flags, ctypes.byref(n_scal), nw, 64)
    want_scal, want_wav = wavelet.bandlimits(L, B, J0, multires, kernel)
    assert ns == len(want_wav)
    assert n_scal.value == want_scal
    assert list(nw[:ns]) == want_wav


@pytest.mark.parametrize("kernel", ["sd", "bspline"])
@pytest.mark.parametrize("L,B,J0", [(128, 3, 2), (256, 2, 1), (100, 3, 0)])
def test_kernel_factors_match_oracle(L, B, J0, kernel):
    lib = _lib.lib()
    J = kernels.jmax(L, B)
    phi, psi = wavelet.tables(L, B, J0, kernel)
    l = np.arange(L)
    to_fac = np.sqrt(4 * np.pi / (2 * l + 1))         # fac = sqrt(4 pi/(2l+1)) Psi_l0
    buf = (ctypes.c_double * L)()
    for j, ref in [(-1, phi)] + list(zip(range(J0, J + 1), psi)):
        assert lib.s2let_wav_kernel(L, B, J0, FLAGS[kernel], j, buf) == _lib.S2LET_OK
        got = np.array(buf[:L])
        assert np.max(np.abs(got - to_fac * ref)) < 1e-11, "j = %d" % j


def test_host_query_argument_errors():
    lib = _lib.lib()
    n = ctypes.c_int()
    nw = (ctypes.c_int * 2)()
    buf = (ctypes.c_double * 8)()
    assert lib.s2let_wav_bandlimits(32, 2, 5, 0, ctypes.byref(n), None, 0) == _lib.S2LET_ERR_ARG   # J0 >= J
    assert lib.s2let_wav_bandlimits(32, 2, 0, 0, ctypes.byref(n), nw, 2) == _lib.S2LET_ERR_ARG     # N_wav too short
    assert lib.s2let_wav_bandlimits(32, 2, 0, 0x1000, ctypes.byref(n), None, 0) == _lib.S2LET_ERR_ARG
    assert lib.s2let_wav_bandlimits(32, 2, 0, 0, ctypes.byref(n), None, 0) == kernels.jmax(32, 2) + 1
    assert lib.s2let_wav_kernel(8, 2, 0, 0, 7, buf) == _lib.S2LET_ERR_ARG                          # j > J
    assert lib.s2let_wav_kernel(8, 2, 0, 0, -2, buf) == _lib.S2LET_ERR_ARG
    assert lib.s2let_wav_kernel(8, 2, 0, 0, -1, None) == _lib.S2LET_ERR_ARG
    # admissibility of the library's own tables (Eq. identity)
    for flags in (0, _lib.S2LET_KERNEL_BSPLINE):
        L, B, J0 = 64, 2, 1
        J = kernels.jmax(L, B)
        tot = np.zeros(L)
        b = (ctypes.c_double * L)()
        for j in [-1] + list(range(J0, J + 1)):
            assert lib.s2let_wav_kernel(L, B, J0, flags, j, b) == 0
            tot += np.array(b[:L]) ** 2
        assert np.max(np.abs(tot - 1.0)) < 1e-13
    assert math.isfinite(tot[0])

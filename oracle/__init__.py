"""ORACLE — test infrastructure only.

A plain, slow FP64 CPU implementation of what the GPU library computes: the
MW-sampled spherical harmonic transforms (Sect. 2.1), the scale-discretised
wavelet kernels (Sect. 2.2) and the axisymmetric wavelet analysis, synthesis
and analysis-adjoint, full-resolution and multiresolution (Sect. 3.1).

Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
bench.py may import this package.  The GPU library neither imports it nor
shares code with it.

Modules: kernels (generating functions, J, band-limits), sht (transforms and
their adjoints), wavelet (analysis / synthesis / adjoint), _clib (builds and
loads the C part, legendre.c).
"""
from . import _clib, kernels, sht, wavelet  # noqa: F401


def build():
    """Compile the oracle's C part (gcc)."""
    return _clib.build()

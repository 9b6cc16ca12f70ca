"""GB300 (sm_103a) implementation of the axisymmetric scale-discretised wavelet
transform on MW-sampled spheres (Leistedt, McEwen, Vandergheynst & Wiaux,
S2LET, A&A 2013).

  build      compiles csrc/ into _build/libs2let_gpu.so (nvcc, sm_103a)
  _lib       ctypes loader of the C ABI (include/s2let_gpu.h)
  s2let      Plan: analysis / synthesis / adjoint / SHTs on torch CUDA tensors
  autograd   torch.autograd.Function whose backward is the adjoint kernel
  inputs     seeded synthetic inputs
"""
__all__ = ["build", "inputs"]

"""The allocation-free inverse transform (s2let_sht_inverse_noalloc) against the
plan-based s2let_sht_inverse, both called through the C ABI.

The entry point exists for callers that cannot allocate device memory
(applications whose device memory is handed out once by a framework or a fixed
budget, plug-ins inside a host program that owns the allocator, real-time hosts
that forbid allocation after start-up); its tables and work buffers are a static
array inside the library.  This file is named to be collected last, so that a
run stopping at the first failure has already run every other test; it passes
alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1211_1680_gb300 import _lib, inputs  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402

TOL = 1e-5   # FP32 tolerance of the parity tests


def _noalloc(L, batch, real, flm_dev):
    shape = (batch, L, 2 * L - 1) if real else (batch, L, 2 * L - 1, 2)
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    flags = _lib.S2LET_PREC_FP32 | (0 if real else _lib.S2LET_COMPLEX)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _lib.lib().s2let_sht_inverse_noalloc(L, batch, flags, ctypes.c_void_p(flm_dev.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), st)
    assert rc == _lib.S2LET_OK, _lib.lib().s2let_strerror(rc)
    return out


@pytest.mark.parametrize("L,batch,real", [(128, 8, True), (33, 3, False), (64, 5, True)])
def test_noalloc_matches_plan_two_calls(L, batch, real):
    plan = Plan(L, 2, 0, batch=batch, real=real, multires=True, precision="fp32")
    for call, seed0 in enumerate((100, 200)):          # two calls in a row, different inputs
        flm = np.stack([inputs.random_flm(L, seed0 + i, real, "white") for i in range(batch)])
        flm_dev = torch.from_numpy(np.stack([flm.real, flm.imag], -1)).to("cuda", torch.float32).contiguous()
        ref = plan.sht_inverse(flm_dev)
        got = _noalloc(L, batch, real, flm_dev)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        err = ((got - ref).abs().max() / ref.abs().max()).item()
        assert err < TOL, (call, err)


def test_noalloc_rejects_sizes_beyond_limits():
    L = _lib.lib()
    dummy = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    assert L.s2let_sht_inverse_noalloc(129, 1, _lib.S2LET_PREC_FP32, p, p, None) == _lib.S2LET_ERR_ARG
    assert L.s2let_sht_inverse_noalloc(32, 9, _lib.S2LET_PREC_FP32, p, p, None) == _lib.S2LET_ERR_ARG
    assert L.s2let_sht_inverse_noalloc(32, 1, _lib.S2LET_PREC_FP64, p, p, None) == _lib.S2LET_ERR_ARG
    assert L.s2let_sht_inverse_noalloc(32, 1, _lib.S2LET_PREC_FP32 | _lib.S2LET_MULTIRES, p, p,
                                       None) == _lib.S2LET_ERR_ARG


def test_noalloc_changes_band_limit_on_a_side_stream():
    """Calls with different band-limits queued back to back on one non-blocking
    stream, with no host synchronisation between them: each call that changes the
    band-limit rewrites the shared tables only after the earlier calls' kernels
    have finished, so every output still matches the plan path."""
    cases = [(64, 4, True), (128, 2, True), (64, 4, True), (40, 3, False)]
    refs, flms = [], []
    for i, (L, batch, real) in enumerate(cases):
        plan = Plan(L, 2, 0, batch=batch, real=real, multires=True, precision="fp32")
        flm = np.stack([inputs.random_flm(L, 300 + 10 * i + b, real, "white") for b in range(batch)])
        flm_dev = torch.from_numpy(np.stack([flm.real, flm.imag], -1)).to("cuda", torch.float32).contiguous()
        refs.append(plan.sht_inverse(flm_dev))
        flms.append(flm_dev)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):       # the outputs are filled and written on the side stream too
        outs = [_noalloc(L, batch, real, flm_dev) for (L, batch, real), flm_dev in zip(cases, flms)]
    side.synchronize()
    for (L, batch, real), got, ref in zip(cases, outs, refs):
        assert torch.isfinite(got).all()
        err = ((got - ref).abs().max() / ref.abs().max()).item()
        assert err < TOL, (L, batch, real, err)

"""Failure paths on the GPU, made without faulting it: a device wait that runs
out (a barrier nothing arrives at, bounded waits), and allocation failures
simulated through the allocator hook (s2let_set_allocator)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sht  # noqa: E402
from paper_1211_1680_gb300 import _lib, inputs, s2let  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402
from tests.gpu_util import TOL, flm_to_dev, from_dev_map, rel_err  # noqa: E402


def _inverse_parity(plan, L, seed=3):
    flm = inputs.random_flm(L, seed, True)
    f = from_dev_map(plan.sht_inverse(flm_to_dev(np.stack([flm] * plan.batch), plan.dtype)), True)
    return rel_err(f, np.stack([sht.inverse(flm, L, real=True)] * plan.batch))


def test_expired_wait_latches_timeout_and_context_survives():
    victim = Plan(16, 2, 0, batch=1, real=True, precision="tf32x3")
    other = Plan(16, 2, 0, batch=1, real=True, precision="tf32x3")
    assert victim.status() == _lib.S2LET_OK
    victim.test_timeout()
    torch.cuda.synchronize()
    assert victim.status() == _lib.S2LET_ERR_TIMEOUT
    assert victim.status() == _lib.S2LET_ERR_TIMEOUT          # latched
    assert other.status() == _lib.S2LET_OK                     # per plan
    # the context is still usable: both plans still transform correctly
    assert _inverse_parity(other, 16) < TOL["tf32x3"]
    assert _inverse_parity(victim, 16) < TOL["tf32x3"]


class _Counting:
    """Allocator hook over PyTorch's caching allocator that fails chosen calls."""

    def __init__(self, fail_at=None, misalign_at=None):
        self.calls = 0
        self.live = {}
        self.fail_at = fail_at
        self.misalign_at = misalign_at

    def alloc(self, n):
        k = self.calls
        self.calls += 1
        if k == self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(n + 256)
        q = p + (16 if k == self.misalign_at else 0)
        self.live[q] = p
        return q

    def release(self, q):
        torch.cuda.caching_allocator_delete(self.live.pop(q))


def _create_with(hook, L=40, prec="tf32x3"):
    s2let.set_allocator(hook.alloc, hook.release)
    try:
        return Plan(L, 2, 1, batch=2, real=True, precision=prec)
    finally:
        s2let.set_allocator()


def test_plan_memory_from_the_hook():
    hook = _Counting()
    plan = _create_with(hook)
    n = hook.calls
    # every table and buffer came from the hook (the temporaries of plan creation
    # went back to it already)
    assert n > 10 and 10 < len(hook.live) < n
    assert _inverse_parity(plan, 40) < TOL["tf32x3"]
    plan.close()
    assert hook.live == {}                          # and went back to it
    # a plan created after the hook was removed does not call it
    Plan(40, 2, 1, batch=2, real=True, precision="tf32x3").close()
    assert hook.calls == n


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_allocation_failures_release_everything(prec):
    total = _Counting()
    _create_with(total, prec=prec).close()
    n = total.calls
    for k in sorted({0, 1, 2, n // 3, n // 2, n - 2, n - 1}):
        hook = _Counting(fail_at=k)
        with pytest.raises(_lib.S2letError) as e:
            _create_with(hook, prec=prec)
        assert e.value.status == _lib.S2LET_ERR_ALLOC, k
        assert hook.live == {}, k                   # nothing leaked
    # a misaligned block is refused like a failed one
    hook = _Counting(misalign_at=n // 2)
    with pytest.raises(_lib.S2letError) as e:
        _create_with(hook, prec=prec)
    assert e.value.status == _lib.S2LET_ERR_ALLOC and hook.live == {}
    # and plans still work afterwards
    assert _inverse_parity(Plan(40, 2, 1, batch=2, real=True, precision=prec), 40) < TOL[prec]

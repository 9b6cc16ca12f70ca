"""GPU parity on the two plain single-map workloads, exactly as stated:

  L = 32, B = 2, J_min = 0, full resolution, one real map, white f_lm, seed 1
  L = 512, B = 2, J_min = 2, multiresolution, one real map, C_l = 1/(l(l+1)), seed 2

Every wavelet map, the scaling map and the reconstruction are compared element
by element with the oracle (normwise max relative error per result): 1e-10 for
FP64 plans, 1e-5 for FP32 and TF32X3 plans.  At L = 512 the round-trip error of
the method grows like L (Sect. 3.3), so this is where the FP64 bound is tightest
among the parity cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sht, wavelet  # noqa: E402
from paper_1211_1680_gb300 import inputs  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402
from tests.gpu_util import TOL, from_dev_map, rel_err, to_dev_map  # noqa: E402

WORKLOADS = {  # name: L, B, J_min, multires, seed, spectrum
    "L32_fullres": (32, 2, 0, False, 1, "white"),
    "L512_multires": (512, 2, 2, True, 2, "cl"),
}

_REF = {}


def _reference(name):
    """Oracle analysis and synthesis of the workload's map (computed once)."""
    if name not in _REF:
        L, B, J0, multires, seed, kind = WORKLOADS[name]
        x = sht.inverse(inputs.random_flm(L, seed, True, kind), L, real=True)
        fw, fs = wavelet.analysis(x, L, B, J0, multires, True)
        _REF[name] = (x, fw, fs)
    return _REF[name]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_workload_parity(name, prec):
    L, B, J0, multires, _, _ = WORKLOADS[name]
    x, fw_ref, fs_ref = _reference(name)
    plan = Plan(L, B, J0, batch=1, real=True, multires=multires, precision=prec)
    tol = TOL[prec]
    fw_d, fs_d = plan.analysis(to_dev_map(x[None], plan.dtype, True))
    views = plan.wavelet_views(fw_d)
    assert len(views) == len(fw_ref)
    for i, view in enumerate(views):
        got = from_dev_map(view, True)[0]
        assert got.shape == fw_ref[i].shape
        assert rel_err(got, fw_ref[i]) < tol, "scale %d" % (J0 + i)
    assert rel_err(from_dev_map(fs_d, True)[0], fs_ref) < tol, "scaling map"
    # reconstruction from the GPU's own wavelet maps, against the input map
    rec = from_dev_map(plan.synthesis(fw_d, fs_d), True)[0]
    assert rel_err(rec, x) < tol, "reconstruction"
    # synthesis of the oracle's wavelet maps, against the oracle's synthesis
    fw_in = torch.cat([to_dev_map(w[None], plan.dtype, True).reshape(-1) for w in fw_ref])
    rec2 = from_dev_map(plan.synthesis(fw_in, to_dev_map(fs_ref[None], plan.dtype, True)), True)[0]
    assert rel_err(rec2, wavelet.synthesis(fw_ref, fs_ref, L, B, J0, multires, True)) < tol, "synthesis"
    assert plan.status() == 0

"""Helpers shared by the GPU tests (not a test module)."""
import numpy as np
import torch


def to_dev_map(x, dtype, real):
    """numpy map(s) -> contiguous CUDA tensor in the library's layout."""
    x = np.asarray(x)
    if not real:
        x = np.stack([x.real, x.imag], axis=-1)
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype).contiguous()


def from_dev_map(t, real):
    a = t.detach().double().cpu().numpy()
    return a if real else a[..., 0] + 1j * a[..., 1]


def flm_to_dev(flm, dtype):
    flm = np.asarray(flm)
    return torch.from_numpy(np.ascontiguousarray(np.stack([flm.real, flm.imag], axis=-1))).to(
        device="cuda", dtype=dtype).contiguous()


def flm_from_dev(t):
    a = t.detach().double().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def rel_err(x, ref):
    """Normwise max relative error: max|x - ref| / max|ref|."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))


TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32x3": 1e-5, "tf32x3s3": 1e-5, "tf32x3rec": 1e-5}


def plan_kwargs(prec):
    """Plan keyword arguments for a precision label of the tests."""
    if prec == "tf32x3s3":
        return {"precision": "tf32x3", "tc_split3": True}
    if prec == "tf32x3rec":                      # Legendre values by the recurrence, no tables
        return {"precision": "tf32x3", "leg_recurrence": True}
    return {"precision": prec}

"""Gradients of the wavelet analysis through the hand-written adjoint kernel:
against central finite differences and against the oracle's explicit adjoint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kernels, sht, wavelet  # noqa: E402
from paper_1211_1680_gb300 import inputs  # noqa: E402
from paper_1211_1680_gb300.autograd import scale_energy_loss, wavelet_analysis  # noqa: E402
from paper_1211_1680_gb300.s2let import Plan  # noqa: E402
from tests.gpu_util import rel_err, to_dev_map  # noqa: E402


def _maps(L, seeds, real=True):
    return np.stack([sht.inverse(inputs.random_flm(L, s, real, "cl"), L, real=real) for s in seeds])


def test_gradient_against_finite_differences():
    """L = 64, FP64, h = 1e-6: 8 random directions and 64 coordinates."""
    L, B, J0 = 64, 2, 2
    plan = Plan(L, B, J0, batch=2, real=True, multires=True, precision="fp64")
    f = to_dev_map(_maps(L, [5, 6]), torch.float64, True).requires_grad_(True)
    loss = scale_energy_loss(f, plan)
    (grad,) = torch.autograd.grad(loss, f)
    h = 1e-6
    fd_noise = 10 * 2.2e-16 * abs(loss.item()) / h     # rounding of the loss difference
    gen = torch.Generator(device="cpu").manual_seed(1)
    with torch.no_grad():
        for _ in range(8):
            d = torch.randn(f.shape, generator=gen, dtype=torch.float64).cuda()
            fd = (scale_energy_loss(f + h * d, plan) - scale_energy_loss(f - h * d, plan)) / (2 * h)
            an = (grad * d).sum()
            assert abs(fd.item() - an.item()) <= 1e-6 * abs(an.item()) + fd_noise
        idx = torch.randperm(f.numel(), generator=gen)[:64]
        flat = f.detach().reshape(-1)
        for i in idx.tolist():
            e = torch.zeros_like(flat)
            e[i] = 1.0
            e = e.view_as(f)
            fd = (scale_energy_loss(f + h * e, plan) - scale_energy_loss(f - h * e, plan)) / (2 * h)
            an = grad.reshape(-1)[i]
            assert abs(fd.item() - an.item()) <= 1e-6 * abs(an.item()) + fd_noise


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5), ("tf32x3", 1e-5)])
def test_gradient_against_oracle_adjoint(prec, tol):
    """L = 256: dLoss/df = A^T (2 w_j W^j) with the oracle's analysis and adjoint."""
    L, B, J0 = 256, 2, 2
    x = _maps(L, [9])
    plan = Plan(L, B, J0, batch=1, real=True, multires=True, precision=prec)
    f = to_dev_map(x, plan.dtype, True).requires_grad_(True)
    loss = scale_energy_loss(f, plan)
    (grad,) = torch.autograd.grad(loss, f)
    fw, fs = wavelet.analysis(x[0], L, B, J0, True, True)
    gw = [2.0 * 2.0 ** -j * w for j, w in zip(range(J0, J0 + len(fw)), fw)]
    ref = wavelet.analysis_adjoint(gw, np.zeros_like(fs), L, B, J0, True, True)
    assert rel_err(grad[0].double().cpu().numpy(), ref) < tol


def test_backward_of_scaling_output_only():
    """Only the scaling map feeds the loss: the gradient is A_scal^T g."""
    L, B, J0 = 32, 2, 1
    plan = Plan(L, B, J0, batch=1, real=True, multires=True, precision="fp64")
    x = _maps(L, [3])
    f = to_dev_map(x, torch.float64, True).requires_grad_(True)
    _, fs = wavelet_analysis(f, plan)
    (grad,) = torch.autograd.grad(fs.sum(), f)
    n_scal, n_wav = kernels.bandlimits(L, B, J0, True)
    ref = wavelet.analysis_adjoint([np.zeros((n, 2 * n - 1)) for n in n_wav], np.ones((n_scal, 2 * n_scal - 1)),
                                   L, B, J0, True, True)
    assert rel_err(grad[0].cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32x3", 1e-5)])
def test_per_scale_recompute_matches_full_backward(prec, tol):
    """The per-scale recomputation gives the loss and gradient of the full
    analysis and adjoint (L = 96, two maps)."""
    from paper_1211_1680_gb300.autograd import scale_energy_loss_recompute
    L, B, J0 = 96, 2, 2
    plan = Plan(L, B, J0, batch=2, real=True, multires=True, precision=prec)
    x = _maps(L, [13, 14])
    f1 = to_dev_map(x, plan.dtype, True).requires_grad_(True)
    l1 = scale_energy_loss(f1, plan)
    (g1,) = torch.autograd.grad(l1, f1)
    f2 = to_dev_map(x, plan.dtype, True).requires_grad_(True)
    l2 = scale_energy_loss_recompute(f2, plan)
    (g2,) = torch.autograd.grad(l2, f2)
    assert abs(l1.item() - l2.item()) <= tol * abs(l1.item())
    assert rel_err(g2.double().cpu().numpy(), g1.double().cpu().numpy()) < tol
    # and against the oracle's explicit adjoint
    fw, fs = wavelet.analysis(x[0], L, B, J0, True, True)
    gw = [2.0 * 2.0 ** -j * w for j, w in zip(range(J0, J0 + len(fw)), fw)]
    ref = wavelet.analysis_adjoint(gw, np.zeros_like(fs), L, B, J0, True, True)
    assert rel_err(g2[0].double().cpu().numpy(), ref) < tol


def test_per_scale_pieces_against_oracle():
    """s2let_wav_scale against the oracle's scale maps, and the transposes of
    s2let_wav_scale and s2let_sht_forward by the dot-product test (FP64, L = 40,
    complex maps, B = 3)."""
    from tests.gpu_util import flm_from_dev, flm_to_dev
    L, B, J0 = 40, 3, 1
    plan = Plan(L, B, J0, batch=1, real=False, multires=True, precision="fp64")
    flm = inputs.random_flm(L, 71, False)
    f = sht.inverse(flm, L)
    fw, fs = wavelet.analysis(f, L, B, J0, True, False)
    fl = flm_to_dev(flm[None], torch.float64)
    for (j, n, _, _), ref in zip(plan.scales, fw):
        w = plan.wav_scale(j, fl)
        got = w[0].cpu().numpy()
        assert rel_err(got[..., 0] + 1j * got[..., 1], ref) < 1e-10, j
    ws = plan.wav_scale(-1, fl)[0].cpu().numpy()
    assert rel_err(ws[..., 0] + 1j * ws[..., 1], fs) < 1e-10
    # <g, S_j x> = <S_j^T g, x> and <y, Fwd f> = <Fwd^T y, f> (real parts of the
    # Euclidean products of the stored arrays)
    for j in (-1, J0, plan.J):
        n = plan.scale_bandlimit(j)
        g = to_dev_map(inputs.random_map((1, n, 2 * n - 1), 90 + j, False), torch.float64, False)
        xs = flm_to_dev(inputs.random_flm(L, 80 + j, False)[None], torch.float64)
        lhs = (g * plan.wav_scale(j, xs)).sum().item()
        glm = torch.zeros_like(xs)
        rhs = (plan.wav_scale_adjoint(j, g, glm) * xs).sum().item()
        assert lhs == pytest.approx(rhs, rel=1e-11), j
    y = flm_to_dev(inputs.random_flm(L, 97, False)[None], torch.float64)
    fd = to_dev_map(inputs.random_map((1, L, 2 * L - 1), 98, False), torch.float64, False)
    lhs = (y * plan.sht_forward(fd)).sum().item()
    rhs = (plan.sht_forward_adjoint(y) * fd).sum().item()
    assert lhs == pytest.approx(rhs, rel=1e-11)

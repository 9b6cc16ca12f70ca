"""Differentiable wavelet analysis: the forward pass is s2let_analysis, the
backward pass is the library's adjoint kernel s2let_adjoint (the transpose of
the analysis operator under the Euclidean inner product of the stored
samples), so gradients with respect to the input maps never go through
PyTorch ops on the transform itself."""
import torch


class WaveletAnalysis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, plan):
        fw, fs = plan.analysis(f.contiguous())
        ctx.plan = plan
        return fw, fs

    @staticmethod
    def backward(ctx, g_wav, g_scal):
        plan = ctx.plan
        if g_wav is None:
            g_wav = torch.zeros(plan.wav_elems, dtype=plan.dtype, device=plan.device)
        if g_scal is None:
            g_scal = torch.zeros(plan.map_shape(plan.N_scal), dtype=plan.dtype, device=plan.device)
        return plan.adjoint(g_wav.contiguous(), g_scal.contiguous()), None


def wavelet_analysis(f, plan):
    """(f_wav, f_scal) = analysis of the maps f, differentiable with respect to f."""
    return WaveletAnalysis.apply(f, plan)


def scale_energy_loss(f, plan, weights=None):
    """sum_j w_j ||W^j||^2 over the wavelet scales (scaling map excluded), summed
    over the batch; default w_j = 2^-j."""
    fw, _ = wavelet_analysis(f, plan)
    loss = f.new_zeros(())
    for (j, _, _, _), view in zip(plan.scales, plan.wavelet_views(fw)):
        w = (2.0 ** -j) if weights is None else weights[j]
        loss = loss + w * (view * view).sum()
    return loss

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


class ScaleEnergyRecompute(torch.autograd.Function):
    """sum_j w_j ||W^j||^2 with one scale in memory at a time: the forward pass
    keeps only f_lm (s2let_sht_forward) and computes each scale's maps, adds their
    energy and drops them; the backward pass recomputes each scale from f_lm
    (s2let_wav_scale), accumulates the transpose of its synthesis applied to
    2 w_j W^j in harmonic space (s2let_wav_scale_adjoint) and applies the
    forward transform's transpose once (s2let_sht_forward_adjoint)."""

    @staticmethod
    def forward(ctx, f, plan, weights):
        flm = plan.sht_forward(f.contiguous())
        loss = f.new_zeros(())
        for (j, _, _, _) in plan.scales:
            w = plan.wav_scale(j, flm)
            loss = loss + weights[j] * (w * w).sum()
            del w
        ctx.plan, ctx.weights = plan, weights
        ctx.save_for_backward(flm)
        return loss

    @staticmethod
    def backward(ctx, gl):
        (flm,) = ctx.saved_tensors
        plan, weights = ctx.plan, ctx.weights
        glm = torch.zeros_like(flm)
        for (j, _, _, _) in plan.scales:
            w = plan.wav_scale(j, flm)
            plan.wav_scale_adjoint(j, (2.0 * weights[j]) * gl * w, glm)
            del w
        return plan.sht_forward_adjoint(glm), None, None


def scale_energy_loss_recompute(f, plan, weights=None):
    """The loss of scale_energy_loss with per-scale recomputation in the backward
    pass (the memory of one scale's maps instead of all of them)."""
    if weights is None:
        weights = {j: 2.0 ** -j for (j, _, _, _) in plan.scales}
    return ScaleEnergyRecompute.apply(f, plan, weights)

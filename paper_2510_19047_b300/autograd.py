"""torch.autograd.Function over tfs_grad_statistic: Upsilon_{N_seg}(theta) with the
adjoint gradient of libtfs as its backward (argument marshalling only)."""
import torch


class StatisticFn(torch.autograd.Function):
    """Upsilon = StatisticFn.apply(theta, ctx, n_seg); theta is a float64 CUDA tensor
    [8, n] (SoA). The forward pass runs the adjoint kernel once and keeps
    d Upsilon / d theta; backward scales it by grad_output."""

    @staticmethod
    def forward(fctx, theta, tfs, n_seg):
        stat, grad = tfs.grad_statistic(theta.detach(), int(n_seg))
        fctx.save_for_backward(grad)
        return stat

    @staticmethod
    def backward(fctx, grad_output):
        (grad,) = fctx.saved_tensors
        return grad * grad_output.unsqueeze(0), None, None


def statistic(theta, tfs, n_seg):
    return StatisticFn.apply(theta, tfs, n_seg)

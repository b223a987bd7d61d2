"""torch.autograd binding of the adjoint gradient (qs_adjoint_gradient).

`circuit_cross_entropy(theta, state, gates, param_index, samples)` returns the
sample cross entropy L = -(1/m) sum_j ln p_theta(x_j) as a 0-d float64 tensor
whose backward gives dL/dtheta from the library's adjoint sweep (computed in
the same library call as the forward value; the sweep needs the forward
state anyway).  `theta` holds the angles of gates[param_index]; the loss and
the gradient are returned on theta's device and in theta's dtype (the
gradient) / float64 (the loss).
"""
import numpy as np
import torch

from . import QS_MODE_FUSED, qs_adjoint_gradient


class _CrossEntropy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, state, gates, param_index, samples, mode):
        g = np.array(gates, copy=True)
        g["theta"][param_index] = theta.detach().cpu().double().numpy()
        loss, grad = qs_adjoint_gradient(state, g, samples, mode=mode)
        ctx.save_for_backward(torch.from_numpy(grad[param_index]).to(device=theta.device, dtype=theta.dtype))
        return torch.tensor(loss, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return gout.to(device=grad.device, dtype=grad.dtype) * grad, None, None, None, None, None


def circuit_cross_entropy(theta, state, gates, param_index, samples, mode=QS_MODE_FUSED):
    return _CrossEntropy.apply(theta, state, gates, np.asarray(param_index), samples, mode)

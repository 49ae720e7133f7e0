"""torch.autograd bindings of the adjoint gradient.

`expval(state, plan, params, obs)` returns E(theta) = <psi(theta)|O|psi(theta)> as
a differentiable scalar tensor: when `params` requires grad, the forward pass calls
sv_grad (forward circuit, lambda = O psi, adjoint sweep) and keeps dE/dtheta for the
backward pass, which only scales it by the incoming gradient; otherwise it calls
sv_run and sv_expval.  `batch_expval(batch, params)` does the same for a Batch (one
E per circuit, the gradient of each circuit's E in its own parameter block).

Every evaluation starts from `psi0` (a host array; default |0...0>), because the
library's calls act on the handle's current state.
"""
import numpy as np
import torch

__all__ = ["expval", "batch_expval"]


def _host(params):
    return np.ascontiguousarray(params.detach().to("cpu", torch.float64).numpy())


class _Expval(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, state, plan, obs, psi0):
        p = _host(params)
        if psi0 is None:
            state.reset()
        else:
            state.set_host(psi0)
        if params.requires_grad:
            e, g = state.grad(plan, p, obs)
            ctx.save_for_backward(torch.as_tensor(g, dtype=params.dtype, device=params.device))
        else:
            state.run(plan, p)
            e = state.expval(obs)
        return torch.tensor(e, dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None


class _BatchExpval(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, batch):
        e, g = batch.run(_host(params))
        ctx.save_for_backward(torch.as_tensor(g, dtype=params.dtype, device=params.device))
        ctx.sizes = list(batch.n_params)
        return torch.as_tensor(e, dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        scale = torch.repeat_interleave(grad_out, torch.as_tensor(ctx.sizes, device=grad_out.device))
        return scale * g, None


def expval(state, plan, params, obs, psi0=None):
    """Differentiable E(theta) for one circuit (see the module docstring)."""
    return _Expval.apply(params, state, plan, obs, psi0)


def batch_expval(batch, params):
    """Differentiable E_i(theta) for every circuit of a Batch (a vector)."""
    return _BatchExpval.apply(params, batch)

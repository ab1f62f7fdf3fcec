"""torch.autograd wrapper: the Tikhonov functional J(eps, sigma) as a
differentiable torch function whose backward pass is the library's adjoint
solve and gradient accumulation (Sec. 3 eq. adjoint_prob, Sec. 4 eq. gradeps).

    loss = ddfd_loss(eps, sigma, problem, eobs)   # eps, sigma: float64 CUDA, free nodes
    loss.backward()                                # eps.grad, sigma.grad from the adjoint

All arithmetic runs in the CUDA library on torch's current stream (the
problem must be created with stream=torch.cuda.current_stream().cuda_stream);
this module only wires the calls.

One handle holds one forward state.  If another loss (or any set_coeffs /
forward call) has used the handle between this loss's forward and its
backward, the handle's generation counter has moved on; backward then
re-runs set_coeffs and the forward from the coefficients this loss saved, so
that its gradient is the one of its own (eps, sigma).
"""
from __future__ import annotations

import torch

from .binding import Problem


class DDFDFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, sig, problem: Problem, eobs):
        e = eps.detach().contiguous()
        s = sig.detach().contiguous()
        problem.set_coeffs_dev(e, s)
        problem.forward_dev(None)
        J = problem.functional_dev(eobs)
        ctx.problem = problem
        ctx.generation = problem.get_info().generation
        ctx.save_for_backward(eobs, e, s)
        return torch.tensor(J, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        eobs, e, s = ctx.saved_tensors
        p = ctx.problem
        if p.get_info().generation != ctx.generation:
            # the handle's forward state belongs to a later call: restore ours
            p.set_coeffs_dev(e, s)
            p.forward_dev(None)
        p.adjoint_dev(eobs)
        ge = torch.empty(p.n_free, dtype=torch.float64, device=eobs.device)
        gs = torch.empty_like(ge)
        p.gradient_dev(ge, gs)
        return grad_out * ge, grad_out * gs, None, None


def ddfd_loss(eps, sig, problem: Problem, eobs):
    """J(eps, sigma) for the given handle and observed data (device tensor in
    the trace layout), differentiable with respect to eps and sigma."""
    return DDFDFunction.apply(eps, sig, problem, eobs)

"""torch.autograd.Function over the library's adjoint gradient.

Forward returns E(theta) = <psi(theta)|H|psi(theta)>. When a gradient will
be needed, the energy and the full gradient come from one sv_grad call
(forward sweep, lambda = H psi, reverse sweep with FP64 gradient reductions
-- all in the CUDA library); otherwise (no_grad, or theta not requiring
grad) only the forward sweep and the expectation run. Backward scales the
stored gradient by the incoming gradient.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np
import torch

from . import StateVector


class AdjointExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, sim: StateVector, gates: Sequence, terms: Sequence):
        th = theta.detach().to("cpu", torch.float64).numpy()
        e, g = sim.grad(gates, th, terms)
        ctx.save_for_backward(torch.from_numpy(np.asarray(g)).to(theta.device, theta.dtype))
        return theta.new_tensor(e)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None


def expectation(theta: torch.Tensor, sim: StateVector, gates: Sequence, terms: Sequence) -> torch.Tensor:
    """Differentiable <H> of the parameterised circuit `gates` at `theta`
    (the energy alone, with no reverse sweep, when no gradient can flow)."""
    if torch.is_grad_enabled() and theta.requires_grad:
        return AdjointExpectation.apply(theta, sim, gates, terms)
    th = theta.detach().to("cpu", torch.float64).numpy()
    return theta.new_tensor(sim.energy(gates, th, terms))

"""torch.autograd.Function around the library (paper, section "PyTorch Model
Support": a model maps positions to an energy; forces come from the backward).

Forward runs staging, neighbors, AEVs and the network forward on the device
and returns the FP64 energy. Backward runs the hand-written network backward
and the AEV-backward force kernel; it reuses the AEVs kept by the forward, or
recomputes them when keep_aev=False (to hold less device memory between the
two passes). The backward returns grad_E * dE/dr, FP32 accumulated in FP64.
"""
from __future__ import annotations

import torch

from .api import System


class MLPEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, system: System, keep_aev: bool = True):
        if not (coords.is_cuda and coords.dtype == torch.float64):
            raise TypeError("coords must be a CUDA float64 tensor [n, 3]")
        c = coords.detach().contiguous()
        E = torch.empty(1, dtype=torch.float64, device=c.device)
        system.forward_device(c, E, keep_aev=keep_aev)
        ctx.system = system
        ctx.save_for_backward(c)
        return E.reshape(())

    @staticmethod
    def backward(ctx, grad_E):
        (c,) = ctx.saved_tensors
        g = torch.empty(c.shape, dtype=torch.float32, device=c.device)
        gE = grad_E.detach().reshape(1).to(torch.float64).contiguous()
        ctx.system.backward_device(c, gE, g)
        return g.to(c.dtype), None, None


def energy(coords, system: System, keep_aev: bool = True):
    """E(coords) as a differentiable scalar (forces = -autograd.grad(E, coords))."""
    return MLPEnergy.apply(coords, system, keep_aev)

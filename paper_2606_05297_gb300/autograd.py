"""The ansatz energy E(theta) of Sec. IV.A/B as a differentiable PyTorch
function: the forward pass calls cvq_energy_and_grad (or its checkpointed
variant for large sectors), which returns the adjoint gradient together with
the energy; backward scales that gradient by the incoming one.  theta may be
a CPU or CUDA float64 tensor; E is a 0-dim float64 tensor on the state's
device."""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import cvq


class AnsatzEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, sector, pool, op_ids, psi0, every, ws):
        th = theta.detach().to("cpu", torch.float64).numpy()
        if every:
            E, g = cvq.energy_and_grad_ckpt(sector, pool, op_ids, th, psi0, int(every), ws=ws)
        else:
            E, g = cvq.energy_and_grad(sector, pool, op_ids, th, psi0, ws=ws)
        ctx.save_for_backward(g.to(theta.device))
        return E.reshape(())

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        return gE.to(g.device) * g, None, None, None, None, None, None


def ansatz_energy(theta: torch.Tensor, sector: "cvq.Sector", pool: "cvq.Pool", op_ids: Sequence[int], psi0,
                  checkpoint_every: Optional[int] = None, ws=None) -> torch.Tensor:
    """E(theta) with autograd support through the adjoint kernels."""
    return AnsatzEnergy.apply(theta, sector, pool, list(op_ids), psi0, checkpoint_every or 0, ws)

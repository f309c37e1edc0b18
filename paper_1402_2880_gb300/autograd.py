"""torch.autograd binding of the SCC energy and its adjoint.

``scc_energy(system, xyz, V0, S0)`` runs the sparse SCF of one cluster
through the C-ABI (sscf_run) and returns the converged energy as a 0-d
tensor; its backward pass returns dE/dxyz and dE/dV0, dE/dS0 from
sscf_gradients (the hand-written adjoint kernels), scaled by the incoming
gradient. Arguments are marshalled to host arrays; every computation runs in
libsscf.
"""
from __future__ import annotations

import numpy as np
import torch

from ._lib import SSCF_FP64, Context


class SCCEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, V0, S0, species, group_of_mol, params, precision, stream):
        p = dict(params)
        p["V0"] = tuple(float(v) for v in V0.detach().cpu().tolist())
        p["S0"] = tuple(float(v) for v in S0.detach().cpu().tolist())
        x = xyz.detach().to("cpu", torch.float64).numpy()
        c = Context(species, x, group_of_mol, p, precision=precision, stream=stream)
        out = c.run(allow_not_converged=True)
        g, gp = c.gradients()
        c.close()
        ctx.save_for_backward(torch.from_numpy(g).to(xyz.device), torch.from_numpy(gp).to(V0.device))
        ctx.converged = out["converged"]
        return torch.tensor(out["energy"], dtype=torch.float64, device=xyz.device)

    @staticmethod
    def backward(ctx, grad_e):
        g, gp = ctx.saved_tensors
        return grad_e * g, grad_e * gp[:4], grad_e * gp[4:], None, None, None, None, None


def scc_energy(system, xyz: torch.Tensor, V0: torch.Tensor, S0: torch.Tensor, params: dict,
               precision: int = SSCF_FP64, stream: int | None = None) -> torch.Tensor:
    """Converged SCC energy of ``system`` at positions ``xyz`` (bohr) with prefactors V0, S0."""
    return SCCEnergy.apply(xyz, V0, S0, np.asarray(system.species, dtype=np.int32),
                           np.asarray(system.group_of_mol, dtype=np.int32), params, precision, stream)

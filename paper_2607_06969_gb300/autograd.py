"""torch.autograd.Function over the C ABI: parameters -> (E_b, F, V_b).

Forward calls nep_set_params and nep_energy_forces_virial; backward calls
nep_param_grad_adjoint with the upstream gradients as the adjoints
(dL/dE_b, dL/dF_i, dL/dV_b), i.e. the vector-Jacobian product of the
paper's training operator (Section 3.2) without autograd caches.
"""
from __future__ import annotations

import torch

from . import binding as nb


class NepRunner:
    """Owns the model, the resident system, its list and both workspaces."""

    def __init__(self, model: nb.Model, dsys: nb.DeviceSystem, nl: nb.NeighborList,
                 ws: nb.Workspace, train_ws: nb.Workspace):
        self.model, self.dsys, self.nl, self.ws, self.train_ws = model, dsys, nl, ws, train_ws


class NepEnergyForcesVirial(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, runner: NepRunner):
        runner.model.set_params(params.detach().contiguous())
        _, force, e_tot, vir = nb.energy_forces_virial(runner.model, runner.dsys, runner.nl, runner.ws)
        ctx.runner = runner
        return e_tot, force, vir

    @staticmethod
    def backward(ctx, g_e, g_f, g_v):
        r = ctx.runner
        B, N = r.dsys.n_cfg, r.dsys.n_atoms
        dev = r.dsys.pos.device
        a_e = (g_e if g_e is not None else torch.zeros(B, device=dev)).to(torch.float64).contiguous()
        lam = (g_f if g_f is not None else torch.zeros(3, N, device=dev)).to(torch.float32).contiguous()
        mu = (g_v if g_v is not None else torch.zeros(B, 9, device=dev)).to(torch.float64).contiguous()
        grad = nb.param_grad_adjoint(r.model, r.dsys, r.nl, r.train_ws, a_e, lam, mu)
        return grad, None


def energy_forces_virial(params: torch.Tensor, runner: NepRunner):
    """Differentiable (E_tot [B] f64, F [3,N] f32, V [B,9] f64)."""
    return NepEnergyForcesVirial.apply(params, runner)

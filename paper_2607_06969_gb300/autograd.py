"""torch.autograd.Function over the C ABI: parameters -> (E_b, F, V_b).

Forward calls nep_set_params and nep_energy_forces_virial; backward calls
nep_param_grad_adjoint with the upstream gradients as the adjoints
(dL/dE_b, dL/dF_i, dL/dV_b), i.e. the vector-Jacobian product of the
paper's training operator (Section 3.2) without autograd caches.

The FP64 Function does the same in double (nep_energy_forces_virial_fp64
and nep_param_grad_adjoint_fp64 with the parameters passed as FP64), so
that torch.autograd.gradcheck can check the operator as Section 3.2 does.
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


class NepRunner64:
    """Model, resident system, list and the FP64 workspaces."""

    def __init__(self, model: nb.Model, dsys: nb.DeviceSystem, nl: nb.NeighborList):
        self.model, self.dsys, self.nl = model, dsys, nl
        self.ws = nb.Workspace64(model, dsys.n_atoms, dsys.n_cfg)
        self.train_ws = nb.Workspace64(model, dsys.n_atoms, dsys.n_cfg, train=True)


class NepEnergyForcesVirial64(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, runner: NepRunner64):
        p = params.detach().contiguous()
        _, force, e_tot, vir = nb.energy_forces_virial_fp64(runner.model, runner.dsys, runner.nl, runner.ws,
                                                            params=p)
        ctx.runner = runner
        ctx.save_for_backward(p)
        return e_tot, force, vir

    @staticmethod
    def backward(ctx, g_e, g_f, g_v):
        r = ctx.runner
        (p,) = ctx.saved_tensors
        B, N = r.dsys.n_cfg, r.dsys.n_atoms
        z = dict(dtype=torch.float64, device=r.dsys.pos.device)
        a_e = (g_e if g_e is not None else torch.zeros(B, **z)).to(torch.float64).contiguous()
        lam = (g_f if g_f is not None else torch.zeros(3, N, **z)).to(torch.float64).contiguous()
        mu = (g_v if g_v is not None else torch.zeros(B, 9, **z)).to(torch.float64).contiguous()
        grad = nb.param_grad_adjoint_fp64(r.model, r.dsys, r.nl, r.train_ws, a_e, lam, mu, params=p)
        return grad, None


def energy_forces_virial_fp64(params: torch.Tensor, runner: NepRunner64):
    """Differentiable (E_tot [B], F [3,N], V [B,9]), all f64, of FP64 parameters."""
    return NepEnergyForcesVirial64.apply(params, runner)

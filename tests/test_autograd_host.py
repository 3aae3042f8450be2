"""The autograd Functions' plumbing on the CPU, with the library calls
replaced by stand-ins: the forward hands the parameters to the model, the
backward passes the upstream gradients as the adjoints in the dtypes and
layouts the C calls take (zeros for outputs the loss does not use), and the
returned vector-Jacobian product reaches the parameters."""
from types import SimpleNamespace

import torch

from paper_2607_06969_gb300 import autograd as AG
from paper_2607_06969_gb300 import binding as nb

N, B, P = 5, 2, 7


def _runner(calls, fp64=False):
    model = SimpleNamespace(set_params=lambda p: calls.append(("set_params", p.dtype, tuple(p.shape))))
    dsys = SimpleNamespace(n_atoms=N, n_cfg=B, pos=torch.zeros(3, N))
    if fp64:
        r = AG.NepRunner64.__new__(AG.NepRunner64)
        r.model, r.dsys, r.nl, r.ws, r.train_ws = model, dsys, None, None, None
    else:
        r = AG.NepRunner(model, dsys, None, None, None)
    return r


def test_fp32_function_adjoints(monkeypatch):
    calls = []
    dt = torch.float32

    def efv(model, dsys, nl, ws, **k):
        p = calls[-1]
        assert p[0] == "set_params"
        return (torch.zeros(N), torch.ones(3, N, dtype=dt), torch.ones(B, dtype=torch.float64),
                torch.ones(B, 9, dtype=torch.float64))

    def adjoint(model, dsys, nl, ws, a_e, lam, mu, **k):
        calls.append(("adjoint", a_e.dtype, tuple(a_e.shape), lam.dtype, tuple(lam.shape), lam.is_contiguous(),
                      mu.dtype, tuple(mu.shape), float(a_e.sum()), float(lam.abs().sum()), float(mu.abs().sum())))
        return torch.arange(P, dtype=torch.float32)

    monkeypatch.setattr(nb, "energy_forces_virial", efv)
    monkeypatch.setattr(nb, "param_grad_adjoint", adjoint)
    params = torch.zeros(P, requires_grad=True)
    E, F, V = AG.energy_forces_virial(params, _runner(calls))
    (2.0 * E.sum()).backward()                        # only E in the loss: lam and mu are zero
    a = calls[-1]
    assert calls[0] == ("set_params", torch.float32, (P,))
    assert a[0] == "adjoint" and a[1:3] == (torch.float64, (B,)) and a[3:6] == (torch.float32, (3, N), True)
    assert a[6:8] == (torch.float64, (B, 9)) and a[8] == 2.0 * B and a[9] == 0.0 and a[10] == 0.0
    assert torch.equal(params.grad, torch.arange(P, dtype=torch.float32))


def test_fp64_function_adjoints(monkeypatch):
    calls = []

    def efv64(model, dsys, nl, ws, params=None, **k):
        calls.append(("efv64", params.dtype, params.requires_grad))
        return (torch.zeros(N, dtype=torch.float64), torch.ones(3, N, dtype=torch.float64),
                torch.ones(B, dtype=torch.float64), torch.ones(B, 9, dtype=torch.float64))

    def adjoint64(model, dsys, nl, ws, a_e, lam, mu, params=None, **k):
        calls.append(("adjoint64", a_e.dtype, lam.dtype, tuple(lam.shape), mu.dtype, params.dtype,
                      float(lam.sum()), float(mu.sum())))
        return torch.ones(P, dtype=torch.float64)

    monkeypatch.setattr(nb, "energy_forces_virial_fp64", efv64)
    monkeypatch.setattr(nb, "param_grad_adjoint_fp64", adjoint64)
    params = torch.zeros(P, dtype=torch.float64, requires_grad=True)
    E, F, V = AG.energy_forces_virial_fp64(params, _runner(calls, fp64=True))
    (F.sum() + 3.0 * V.sum()).backward()              # E unused: a_e is zero
    assert calls[0] == ("efv64", torch.float64, False)   # the forward sees detached parameters
    a = calls[-1]
    assert a[:6] == ("adjoint64", torch.float64, torch.float64, (3, N), torch.float64, torch.float64)
    assert a[6] == 3 * N and a[7] == 3.0 * 9 * B
    assert torch.equal(params.grad, torch.ones(P, dtype=torch.float64))

"""FP64 training operator (nep_param_grad_fp64, nep_param_grad_adjoint_fp64
and the FP64 autograd Function) against the FP64 oracle.

The oracle's complex-step gradient is exact to rounding, and the GPU path
computes the same quantities in double.  Both sum ~10^4 terms per
component, so they agree to ~1e-13 relative.  The bar of 1e-9 (relative L2
over the checked components) leaves a wide margin, while a dropped term or
a wrong sign moves the result by orders of magnitude more.  At sizes where
the oracle is too slow, the FP64 gradient is compared with the FP32 GPU
gradient at the FP32 bar (relative L2 1e-4).
"""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 1e-4
W = (1.0, 1.0, 0.1)
TINY = I.Hyper(n_rad=3, n_ang=2, k_rad=4, k_ang=3, n_hidden=4, rc_rad=5.0, rc_ang=4.0)


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(b))


class Case64:
    """A batch with teacher labels from the oracle; FP64 student weights that
    FP32 cannot hold (seed-1 weights with a relative jitter of 1e-7)."""

    def __init__(self, h, s, cap=112, cap_ang=56):
        self.h, self.s = h, s
        self.p32 = s.pos32()
        self.box64 = s.box.astype(np.float32).astype(np.float64)
        self.pairs = O.neighbor_pairs(self.p32, s.box, s.atom_off, h.rc_rad)
        teacher = I.init_params(h, seed=I.SEED_TEACHER)
        lab = O.energy_forces_virial(h, teacher, self.p32.astype(np.float64), s.types, self.box64,
                                     s.atom_off, self.pairs)
        self.E, self.F, self.V = lab["Etot"], lab["F"], lab["V"].reshape(-1, 9)
        rng = np.random.default_rng(21)
        self.theta = I.init_params(h) * (1.0 + 1e-7 * rng.standard_normal(h.n_params))
        self.cap, self.cap_ang = cap, cap_ang

    def oracle_loss(self, theta, mode=0):
        return O.loss_value(self.h, theta, self.p32.astype(np.float64), self.s.types, self.box64,
                            self.s.atom_off, self.pairs, self.E, self.F, self.V, W, mode)

    def gpu(self, nb):
        import torch
        s = self.s
        g = dict(model=nb.Model(self.h, self.theta.astype(np.float32)), dsys=nb.DeviceSystem.from_inputs(s),
                 nl=nb.NeighborList(s.n_atoms, self.cap, self.cap_ang))
        ws = nb.Workspace(g["model"], s.n_atoms, s.n_cfg, self.cap, self.cap_ang)
        nb.neighbors(g["model"], g["dsys"], g["nl"], 0.0, ws)
        assert nb.check_list(g["nl"]) == nb.NEP_OK
        g["tws"] = nb.Workspace64(g["model"], s.n_atoms, s.n_cfg, train=True)
        dev = dict(dtype=torch.float64, device="cuda")
        g["p64"] = torch.tensor(self.theta, **dev)
        g["E"] = torch.tensor(self.E, **dev)
        g["F"] = torch.tensor(np.ascontiguousarray(self.F.T), **dev)
        g["V"] = torch.tensor(np.ascontiguousarray(self.V), **dev)
        return g

    def gpu_grad(self, nb, g, mode=0):
        grad, loss = nb.param_grad_fp64(g["model"], g["dsys"], g["nl"], g["tws"], g["E"], g["F"], g["V"], W,
                                        mode, params=g["p64"])
        return grad.cpu().numpy(), float(loss.item())


@pytest.fixture(scope="module")
def tiny64():
    return Case64(TINY, I.packing_batch([24, 31, 40], tag=91))


@pytest.mark.parametrize("mode", [0, 1])
def test_fp64_full_gradient_tiny_model(nb, tiny64, mode):
    """Every one of the 345 parameters against the complex-step gradient."""
    c = tiny64
    g = c.gpu(nb)
    grad, loss = c.gpu_grad(nb, g, mode)
    ref = O.complex_step_grad(lambda t: c.oracle_loss(t, mode), c.theta, np.arange(c.h.n_params))
    assert rel_l2(grad, ref) <= TOL64
    # the loss squares E_b - E_label with |E_b| >> |E_b - E_label|: the two
    # sides' last-bit differences in E_b are amplified by that ratio
    assert abs(loss - c.oracle_loss(c.theta, mode)) <= TOL64 * abs(loss)


@pytest.mark.parametrize("hname", ["HYPER_SMALL", "HYPER_TABLE2", "HYPER_LARGE"])
def test_fp64_sampled_gradient(nb, hname):
    """The 38-30-1 model with 4-body terms, the Table 2 model (2+3-body,
    n_A = 8) and the 52-64-1 model (n_R = 12, n_A = 8): parameters sampled
    from every block (W0, b0, w1, b1, cR, cA) of every species."""
    h = getattr(I, hname)
    c = Case64(h, I.packing_batch([24, 57, 100], tag=92))
    g = c.gpu(nb)
    grad, _ = c.gpu_grad(nb, g)
    D, H, T = O.descriptor_dim(h), h.n_hidden, h.n_types
    stride = H * D + 2 * H + 1
    idx = []
    rng = np.random.default_rng(22)
    for t in range(T):
        base = t * stride
        idx += list(base + rng.choice(H * D, 6, replace=False))
        idx += [base + H * D + int(rng.integers(H)), base + H * D + H + int(rng.integers(H)), base + stride - 1]
    off_cR = T * stride
    nR = T * T * h.n_rad * h.k_rad
    idx += list(off_cR + rng.choice(nR, 12, replace=False))
    idx += list(off_cR + nR + rng.choice(h.n_params - off_cR - nR, 12, replace=False))
    idx = np.array(sorted(set(int(i) for i in idx)))
    ref = O.complex_step_grad(c.oracle_loss, c.theta, idx)
    assert rel_l2(grad[idx], ref) <= TOL64


def test_fp64_gradcheck_autograd(nb):
    """torch.autograd.gradcheck of the FP64 Function (parameters -> E, F, V):
    central differences in double against the analytic vector-Jacobian
    products, for every parameter and every output."""
    import torch
    from paper_2607_06969_gb300 import autograd as AG
    h = TINY
    s = I.packing_batch([10, 14], tag=95)
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 112, 56)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, 112, 56)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    runner = AG.NepRunner64(model, dsys, nl)
    p = torch.tensor(I.init_params(h), dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: AG.energy_forces_virial_fp64(x, runner), (p,),
                                    eps=1e-6, atol=1e-7, rtol=1e-5)


def test_fp64_adjoint_call_matches_loss_call_and_repeats(nb, tiny64):
    """The loss call equals the adjoint call fed with the loss adjoints
    (formed here from the FP64 E, F, V), and repeats bitwise."""
    import torch
    c = tiny64
    g = c.gpu(nb)
    grad, _ = c.gpu_grad(nb, g)
    grad2, _ = c.gpu_grad(nb, g)
    assert np.array_equal(grad, grad2)
    ws = nb.Workspace64(g["model"], c.s.n_atoms, c.s.n_cfg)
    _, F, E, V = nb.energy_forces_virial_fp64(g["model"], g["dsys"], g["nl"], ws, params=g["p64"])
    n = torch.tensor(np.diff(c.s.atom_off), dtype=torch.float64, device="cuda")
    B = c.s.n_cfg
    a_e = (2.0 * W[0] * (E - g["E"]) / n ** 2 / B).contiguous()
    cfg = torch.tensor(c.s.cfg_of_atom(), device="cuda", dtype=torch.long)
    lam = (2.0 * W[1] * (F - g["F"]) / (3.0 * n[cfg] * B)).contiguous()
    mu = (2.0 * W[2] * (V - g["V"]) / (9.0 * n[:, None] ** 2) / B).contiguous()
    ga = nb.param_grad_adjoint_fp64(g["model"], g["dsys"], g["nl"], g["tws"], a_e, lam, mu,
                                    params=g["p64"]).cpu().numpy()
    # adjoints formed in another rounding order; the gradient sums terms of
    # both signs, which amplifies that difference
    assert rel_l2(ga, grad) <= TOL64


@pytest.mark.parametrize("ncell", [14, 28])
def test_fp64_gradient_at_scale_against_fp32(nb, ncell):
    """19,757 atoms (8 lanes per atom) and 158,054 atoms (one thread per
    atom): the FP64 gradient against the FP32 GPU gradient at the FP32 bar,
    with FP32-representable weights so that both see the same model."""
    import torch
    h = I.HYPER_SMALL
    s = I.rocksalt(ncell, vacancy=0.2, tag=6)
    th32 = I.init_params(h).astype(np.float32)
    teacher = nb.Model(h, I.init_params(h, seed=I.SEED_TEACHER).astype(np.float32))
    model = nb.Model(h, th32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 112, 56, shifts=False)
    ws = nb.Workspace(model, s.n_atoms, 1, 112, 56, train=True)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    # labels: the teacher in FP32, perturbed so that every loss term is active
    _, F, E, V = nb.energy_forces_virial(teacher, dsys, nl, ws)
    F = (F + 0.01).contiguous()
    g32, l32 = nb.param_grad(model, dsys, nl, ws, E, F, V, W, 0)
    ws64 = nb.Workspace64(model, s.n_atoms, 1, train=True)
    g64, l64 = nb.param_grad_fp64(model, dsys, nl, ws64, E, F.double().contiguous(), V, W, 0)
    g32, g64 = g32.cpu().numpy().astype(np.float64), g64.cpu().numpy()
    assert rel_l2(g32, g64) <= TOL32
    assert abs(float(l32.item()) - float(l64.item())) <= 1e-4 * abs(float(l64.item()))
    del ws64, ws
    torch.cuda.synchronize()

"""Training backward (nep_param_grad, nep_param_grad_adjoint, the autograd
Function) against the FP64 oracle's complex-step gradient and central
differences.  Bar: relative L2 error of the gradient <= 1e-4."""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_G = 1e-4
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


class Case:
    """A batch, its oracle neighbour pairs and teacher labels (oracle, FP64)."""

    def __init__(self, h, s, cap=96, cap_ang=48):
        self.h, self.s, self.cap, self.cap_ang = h, s, cap, cap_ang
        self.p32 = s.pos32()
        self.box64 = s.box.astype(np.float32).astype(np.float64)
        self.pairs = O.neighbor_pairs(self.p32, s.box, s.atom_off, h.rc_rad)
        teacher = I.init_params(h, seed=I.SEED_TEACHER).astype(np.float32).astype(np.float64)
        lab = O.energy_forces_virial(h, teacher, self.p32.astype(np.float64), s.types, self.box64,
                                     s.atom_off, self.pairs)
        self.E, self.F, self.V = lab["Etot"], lab["F"], lab["V"].reshape(-1, 9)

    def oracle_loss(self, theta, mode=0):
        return O.loss_value(self.h, theta, self.p32.astype(np.float64), self.s.types, self.box64,
                            self.s.atom_off, self.pairs, self.E, self.F, self.V, W, mode)

    def oracle_grad(self, theta, idx, mode=0):
        return O.complex_step_grad(lambda t: self.oracle_loss(t, mode), theta, idx)

    def gpu(self, nb, theta32):
        import torch
        s = self.s
        g = dict(model=nb.Model(self.h, theta32), dsys=nb.DeviceSystem.from_inputs(s),
                 nl=nb.NeighborList(s.n_atoms, self.cap, self.cap_ang))
        g["ws"] = nb.Workspace(g["model"], s.n_atoms, s.n_cfg, self.cap, self.cap_ang)
        g["tws"] = nb.Workspace(g["model"], s.n_atoms, s.n_cfg, self.cap, self.cap_ang, train=True)
        nb.neighbors(g["model"], g["dsys"], g["nl"], 0.0, g["ws"])
        assert nb.check_list(g["nl"]) == nb.NEP_OK
        g["E"] = torch.tensor(self.E, dtype=torch.float64, device="cuda")
        g["F"] = torch.tensor(np.ascontiguousarray(self.F.T), dtype=torch.float32, device="cuda")
        g["V"] = torch.tensor(self.V, dtype=torch.float64, device="cuda")
        return g

    def gpu_grad(self, nb, g, mode=0):
        grad, loss = nb.param_grad(g["model"], g["dsys"], g["nl"], g["tws"], g["E"], g["F"], g["V"],
                                   W, mode)
        assert nb.check_list(g["nl"]) == nb.NEP_OK
        return grad.cpu().numpy().astype(np.float64), float(loss.item())


@pytest.fixture(scope="module")
def tiny_case():
    return Case(TINY, I.packing_batch([24, 31, 40], tag=91))


@pytest.fixture(scope="module")
def small_case():
    return Case(I.HYPER_SMALL, I.packing_batch([24, 57, 100], tag=92))


@pytest.mark.parametrize("mode", [0, 1])
def test_full_gradient_small_model(nb, tiny_case, mode):
    c = tiny_case
    th32 = I.init_params(c.h).astype(np.float32)
    th = th32.astype(np.float64)
    g = c.gpu(nb, th32)
    grad, loss = c.gpu_grad(nb, g, mode)
    want = c.oracle_grad(th, list(range(th.size)), mode)
    assert rel_l2(grad, want) <= TOL_G
    assert abs(loss - c.oracle_loss(th, mode)) <= 1e-5 * abs(c.oracle_loss(th, mode))


def test_sampled_gradient_216_atom_model(nb, small_case):
    c = small_case
    th32 = I.init_params(c.h).astype(np.float32)
    th = th32.astype(np.float64)
    grad, _ = c.gpu_grad(nb, c.gpu(nb, th32))
    P = th.size
    rng = np.random.default_rng(0)
    idx = sorted(set(rng.choice(3000, 40, replace=False).tolist()     # network weights
                     + (3420 + rng.choice(P - 3420, 60, replace=False)).tolist()))   # biases and c
    want = c.oracle_grad(th, idx)
    assert rel_l2(grad[idx], want) <= TOL_G


def block_sample(h, rng, per=6):
    """Parameter indices from every block (W0, b0, w1, b1 of each species,
    then cR and cA)."""
    D = O.descriptor_dim(h)
    H, T = h.n_hidden, h.n_types
    stride = H * D + 2 * H + 1
    idx = []
    for t in range(T):
        base = t * stride
        idx += list(base + rng.choice(H * D, per, replace=False))
        idx += [base + H * D + int(rng.integers(H)), base + H * D + H + int(rng.integers(H)), base + stride - 1]
    off_cR = T * stride
    nR = T * T * h.n_rad * h.k_rad
    idx += list(off_cR + rng.choice(nR, 2 * per, replace=False))
    idx += list(off_cR + nR + rng.choice(h.n_params - off_cR - nR, 2 * per, replace=False))
    return sorted(set(int(i) for i in idx))


@pytest.mark.parametrize("hname", ["HYPER_TABLE2", "HYPER_LARGE"])
def test_sampled_gradient_other_compiled_models(nb, hname):
    """The Table 2 model (2+3-body, n_A = 8) and the 52-64-1 model
    (n_R = 12, n_A = 8, 4-body): the training kernels of their compiled sets."""
    h = getattr(I, hname)
    c = Case(h, I.packing_batch([24, 57], tag=96))
    th32 = I.init_params(h).astype(np.float32)
    th = th32.astype(np.float64)
    grad, loss = c.gpu_grad(nb, c.gpu(nb, th32))
    idx = block_sample(h, np.random.default_rng(30))
    want = c.oracle_grad(th, idx)
    assert rel_l2(grad[idx], want) <= TOL_G
    assert abs(loss - c.oracle_loss(th)) <= 1e-5 * abs(c.oracle_loss(th))


def test_gradient_against_central_differences(nb, small_case):
    c = small_case
    th32 = I.init_params(c.h).astype(np.float32)
    th = th32.astype(np.float64)
    grad, _ = c.gpu_grad(nb, c.gpu(nb, th32))
    idx = [5, 700, 1500, 3450, 3500, 3650, 3900, 4200, 4500, 4600]
    h = 1e-4
    fd = []
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd.append((c.oracle_loss(tp) - c.oracle_loss(tm)) / (2 * h))
    assert rel_l2(grad[idx], fd) <= TOL_G


def test_adjoint_call_and_autograd_agree_with_loss_call(nb, small_case):
    import torch
    from paper_2607_06969_gb300 import autograd as NA
    c = small_case
    th32 = I.init_params(c.h).astype(np.float32)
    g = c.gpu(nb, th32)
    grad, _ = c.gpu_grad(nb, g)
    runner = NA.NepRunner(g["model"], g["dsys"], g["nl"], g["ws"], g["tws"])
    params = torch.tensor(th32, device="cuda", requires_grad=True)
    e_tot, force, vir = NA.energy_forces_virial(params, runner)
    Nb = torch.tensor(np.diff(c.s.atom_off), dtype=torch.float64, device="cuda")
    cfg = torch.tensor(c.s.cfg_of_atom(), device="cuda")
    B = c.s.n_cfg
    dF2 = ((force - g["F"]) ** 2).sum(0).to(torch.float64)
    sF = torch.zeros(B, dtype=torch.float64, device="cuda").index_add_(0, cfg, dF2)
    loss = (W[0] * ((e_tot - g["E"]) / Nb) ** 2 + W[1] * sF / (3 * Nb)
            + W[2] * (((vir - g["V"]) / Nb[:, None]) ** 2).sum(1) / 9).mean()
    loss.backward()
    assert rel_l2(params.grad.cpu().numpy(), grad) <= 1e-5


def test_gradient_is_deterministic(nb, small_case):
    c = small_case
    th32 = I.init_params(c.h).astype(np.float32)
    g = c.gpu(nb, th32)
    a, la = c.gpu_grad(nb, g)
    b, lb = c.gpu_grad(nb, g)
    assert np.array_equal(a, b) and la == lb


@pytest.mark.slow
def test_train128_full_batch(nb):
    """The 128-configuration batch (N ~ U{24..512}): sampled components
    against the oracle, and additivity over configurations (the batch
    gradient is the mean of the per-configuration gradients)."""
    import torch
    s, h = I.workload_train128()
    c = Case(h, s, cap=112, cap_ang=56)
    th32 = I.init_params(h).astype(np.float32)
    th = th32.astype(np.float64)
    g = c.gpu(nb, th32)
    grad, loss = c.gpu_grad(nb, g)
    idx = [1200, 3500, 4300]
    want = c.oracle_grad(th, idx)
    assert rel_l2(grad[idx], want) <= TOL_G
    # additivity, on the GPU path itself, one configuration at a time
    acc = np.zeros_like(grad)
    for b in range(s.n_cfg):
        a0, a1 = s.atom_off[b], s.atom_off[b + 1]
        sb = I.System(pos=s.pos[a0:a1], types=s.types[a0:a1], box=s.box[b:b + 1],
                      atom_off=np.array([0, a1 - a0]))
        m = nb.Model(h, th32)
        d = nb.DeviceSystem.from_inputs(sb)
        nl = nb.NeighborList(sb.n_atoms, 112, 56)
        ws = nb.Workspace(m, sb.n_atoms, 1, 112, 56, train=True)
        nb.neighbors(m, d, nl, 0.0, ws)
        E = torch.tensor(c.E[b:b + 1], dtype=torch.float64, device="cuda")
        F = torch.tensor(np.ascontiguousarray(c.F[a0:a1].T), dtype=torch.float32, device="cuda")
        V = torch.tensor(c.V[b:b + 1], dtype=torch.float64, device="cuda")
        gb, _ = nb.param_grad(m, d, nl, ws, E, F, V, W, 0)
        acc += gb.cpu().numpy()
    assert rel_l2(grad, acc / s.n_cfg) <= 1e-5

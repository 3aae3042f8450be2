"""Mixed-precision network (FP16 / BF16 tensor-core MLP, FP32 descriptors and
forces, FP64 sums) against the FP64 oracle.  Bar: force RMS <= 2 meV/A and
|dE_tot|/N <= 0.5 meV/atom."""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_FRMS, TOL_E_ATOM = 2e-3, 5e-4


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


def run(nb, h, th32, s, precision, cap=96, cap_ang=40):
    model = nb.Model(h, th32, precision=precision)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, cap, cap_ang)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    return e.cpu().numpy(), f.cpu().numpy().T, et.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("hname", ["small", "large"])
def test_mixed_against_oracle(nb, precision, hname):
    h = I.HYPER_SMALL if hname == "small" else I.HYPER_LARGE
    s = I.rocksalt(3, tag=0) if hname == "small" else I.rocksalt(4, vacancy=0.2, tag=63)
    th32 = I.init_params(h).astype(np.float32)
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    ref = O.energy_forces_virial(h, th32.astype(np.float64), p32.astype(np.float64), s.types,
                                 s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)
    e, f, et, v = run(nb, h, th32, s, precision)
    frms = np.sqrt(np.mean((f - ref["F"]) ** 2))
    de = abs(et[0] - ref["Etot"][0]) / s.n_atoms
    assert frms <= TOL_FRMS, frms
    assert de <= TOL_E_ATOM, de
    # the FP32 path on the same system is much closer
    e32, f32, et32, _ = run(nb, h, th32, s, 0)
    assert np.sqrt(np.mean((f32 - ref["F"]) ** 2)) < 1e-5


def test_mixed_training_is_rejected(nb):
    h = I.HYPER_SMALL
    s, _ = I.workload_cell216()
    model = nb.Model(h, I.init_params(h).astype(np.float32), precision=1)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 96, 40)
    ws = nb.Workspace(model, s.n_atoms, 1, 96, 40, train=True)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    import torch
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(nb.NepError) as err:
        nb.param_grad(model, dsys, nl, ws, z, torch.zeros(3, s.n_atoms, device="cuda"),
                      torch.zeros(1, 9, dtype=torch.float64, device="cuda"))
    assert err.value.status == nb.NEP_ERR_UNSUPPORTED

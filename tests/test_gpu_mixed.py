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


def run(nb, h, th32, s, precision, cap=96, cap_ang=40, variant=-1):
    model = nb.Model(h, th32, precision=precision)
    nb.set_variant(model, variant)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, cap, cap_ang)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    return e.cpu().numpy(), f.cpu().numpy().T, et.cpu().numpy(), v.cpu().numpy()


TINY = I.Hyper(n_rad=3, n_ang=2, k_rad=4, k_ang=3, n_hidden=4, rc_rad=5.0, rc_ang=4.0)
MODELS = dict(small=I.HYPER_SMALL, large=I.HYPER_LARGE, tiny=TINY, table2=I.HYPER_TABLE2)
_REF = {}


def system(hname):
    # 216 atoms (two tiles of 128, ragged), 460 atoms (four tiles), uneven batch
    if hname == "large":
        return I.rocksalt(4, vacancy=0.2, tag=63)
    if hname == "table2":
        return I.packing_batch([24, 77, 130], tag=71)
    return I.rocksalt(3, tag=0)


def reference(hname):
    if hname not in _REF:
        h = MODELS[hname]
        s = system(hname)
        th32 = I.init_params(h).astype(np.float32)
        p32 = s.pos32()
        pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
        _REF[hname] = (s, th32, O.energy_forces_virial(h, th32.astype(np.float64), p32.astype(np.float64),
                                                       s.types, s.box.astype(np.float32).astype(np.float64),
                                                       s.atom_off, pairs))
    return _REF[hname]


def check_mixed(e, f, et, ref, s):
    frms = np.sqrt(np.mean((f - ref["F"]) ** 2))
    Nb = np.diff(s.atom_off)
    de = np.abs(et - ref["Etot"]) / np.maximum(Nb, 1)
    assert frms <= TOL_FRMS, frms
    assert de.max() <= TOL_E_ATOM, de


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("hname", ["small", "large", "tiny", "table2"])
def test_mixed_against_oracle(nb, precision, hname):
    h = MODELS[hname]
    s, th32, ref = reference(hname)
    e, f, et, v = run(nb, h, th32, s, precision)
    check_mixed(e, f, et, ref, s)
    # the FP32 path on the same system is much closer; per-atom energies of the
    # two differ only by the 16-bit rounding of q and W0 (a wrong row, column
    # or species block would show up as O(0.1 eV))
    e32, f32, et32, _ = run(nb, h, th32, s, 0)
    assert np.sqrt(np.mean((f32 - ref["F"]) ** 2)) < 1e-5
    assert np.abs(e - e32).max() < (5e-3 if precision == 1 else 3e-2)


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("hname", ["small", "large"])
def test_mixed_every_variant(nb, hname, variant):
    """S_nlm in tensor memory (variant 0) or in global memory (1, 2)."""
    h = MODELS[hname]
    s, th32, ref = reference(hname)
    e, f, et, v = run(nb, h, th32, s, 1, variant=variant)
    check_mixed(e, f, et, ref, s)
    e0, f0, _, _ = run(nb, h, th32, s, 1, variant=0)
    assert np.abs(e - e0).max() <= 1e-6          # the network path is the same in every variant
    assert np.abs(f - f0).max() <= 1e-5


def test_mixed_single_species_and_single_atom(nb):
    """Tiles where only one species is present (the other GEMM1 rounds are
    skipped) and a one-atom configuration (a tile of one valid row)."""
    h = I.HYPER_SMALL
    s0 = I.packing_batch([40, 1, 150], tag=72)
    types = s0.types.copy()
    types[s0.atom_off[2]:] = 2                    # third configuration: Te only
    s = I.System(pos=s0.pos, types=types, box=s0.box, atom_off=s0.atom_off)
    th32 = I.init_params(h).astype(np.float32)
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    ref = O.energy_forces_virial(h, th32.astype(np.float64), p32.astype(np.float64), s.types,
                                 s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)
    for precision in (1, 2):
        e, f, et, v = run(nb, h, th32, s, precision, cap=160, cap_ang=64)
        check_mixed(e, f, et, ref, s)


def test_mixed_hidden_width_limit(nb):
    h = I.Hyper(n_rad=8, n_ang=6, k_rad=8, k_ang=8, n_hidden=65, rc_rad=7.0, rc_ang=5.0)
    with pytest.raises(nb.NepError) as err:
        nb.Model(h, I.init_params(h).astype(np.float32), precision=1)
    assert err.value.status == nb.NEP_ERR_UNSUPPORTED
    nb.Model(h, I.init_params(h).astype(np.float32), precision=0)


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

"""The generic FP32 path: shapes with no compiled kernel set (runtime
hyper-parameters within n <= 16, K <= 16) against the FP64 oracle at the FP32
parity bars of test_gpu_parity.py (E_i 1e-6 eV, F 1e-4 eV/A, E_tot 1e-6 eV
and V 1e-5 eV per atom of the configuration), through nep_energy_forces_virial,
its owned-prefix and allocation-free forms and a few nep_md_step calls; the
FP32 training calls are refused and the FP64 gradient serves the shape."""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_E, TOL_F, TOL_ET, TOL_V = 1e-6, 1e-4, 1e-6, 1e-5
SHAPES = {
    "r5a3k6k5_4body": I.Hyper(n_types=3, n_rad=5, n_ang=3, k_rad=6, k_ang=5, has_4body=1, n_hidden=7,
                              rc_rad=7.0, rc_ang=5.0),
    "r11a7k10k9_two_species": I.Hyper(n_types=2, n_rad=11, n_ang=7, k_rad=10, k_ang=9, has_4body=0,
                                      n_hidden=20, rc_rad=6.0, rc_ang=4.5),
}


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


def system_for(h, tag):
    s = I.packing_batch([24, 130, 400], tag=tag)
    if h.n_types < 3:
        s = I.System(pos=s.pos, types=(s.types % h.n_types).astype(np.int32), box=s.box, atom_off=s.atom_off,
                     meta=s.meta)
    return s


def oracle_eval(h, th32, s):
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    return O.energy_forces_virial(h, th32.astype(np.float64), p32.astype(np.float64), s.types,
                                  s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)


def check(out, ref, s):
    e, f, et, v = [t.cpu().numpy() for t in out]
    Nb = np.maximum(np.diff(s.atom_off), 1)
    assert np.abs(e - ref["E"]).max() <= TOL_E
    assert np.abs(f.T - ref["F"]).max() <= TOL_F
    assert np.all(np.abs(et - ref["Etot"]) <= TOL_ET * Nb)
    assert np.all(np.abs(v.reshape(-1, 3, 3) - ref["V"]).reshape(-1, 9).max(1) <= TOL_V * Nb)


@pytest.mark.parametrize("name", list(SHAPES))
def test_generic_shapes_against_oracle(nb, name):
    import ctypes
    h = SHAPES[name]
    assert nb.lib().nep_supported(ctypes.byref(nb.hparams_of(h))) == 2
    th32 = I.init_params(h, seed=13).astype(np.float32)
    s = system_for(h, 41)
    model = nb.Model(h, th32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 160, 64, shifts=True)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, 160, 64)
    nb.neighbors(model, dsys, nl, 1.0, ws)
    out = nb.energy_forces_virial(model, dsys, nl, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    ref = oracle_eval(h, th32, s)
    check(out, ref, s)
    # the allocation-free form gives the same bits
    if ws.bytes <= nb.NOALLOC_SCRATCH_BYTES:
        out2 = nb.energy_forces_virial_noalloc(model, dsys, nl)
        for x, y in zip(out, out2):
            assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_generic_owned_prefix_and_md(nb):
    import ctypes

    import torch
    h = SHAPES["r5a3k6k5_4body"]
    th32 = I.init_params(h, seed=17).astype(np.float32)
    s = I.packing_batch([300], tag=43)
    model = nb.Model(h, th32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 160, 64, shifts=True)
    ws = nb.Workspace(model, s.n_atoms, 1, 160, 64)
    nb.neighbors(model, dsys, nl, 1.0, ws)
    e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
    # energy and virial summed over an owned prefix
    n_owned = 120
    e2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    v2 = torch.zeros(1, 9, dtype=torch.float64, device="cuda")
    f2 = torch.zeros_like(f)
    nb.check(nb.lib().nep_energy_forces_virial_owned(
        model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c), n_owned, None, nb._ptr(f2), nb._ptr(e2),
        nb._ptr(v2), ws.ptr, ws.bytes, nb._stream()), "owned")
    assert abs(e2.item() - e[:n_owned].double().sum().item()) <= 1e-9 * n_owned + 1e-6
    assert torch.equal(f2, f)
    # three MD steps (a rebuild at the first) against the oracle's integrator
    m32 = I.MASSES.astype(np.float32)
    v0 = I.maxwell_boltzmann(s.types, 900.0, atom_off=s.atom_off).astype(np.float32)
    vel = torch.from_numpy(np.ascontiguousarray(v0.T)).cuda()
    for k in range(3):
        nb.md_step(model, dsys, nl, vel, f, et, v, m32, 2.0, 1.0, k == 0, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    r = O.velocity_verlet(h, th32.astype(np.float64), s.pos32().astype(np.float64), v0.astype(np.float64),
                          s.types, s.box.astype(np.float32).astype(np.float64), s.atom_off,
                          m32.astype(np.float64), 2.0, 3)
    L = s.box[0]
    d = dsys.pos.cpu().numpy().T - r["pos"]
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 1e-4
    assert np.abs(vel.cpu().numpy().T - r["vel"]).max() <= 1e-6


def test_generic_training_calls(nb):
    """FP32 training and tuning are refused for a generic shape; the FP64
    gradient serves it (sampled against the oracle's complex-step gradient)."""
    import torch
    h = SHAPES["r5a3k6k5_4body"]
    th32 = I.init_params(h, seed=19).astype(np.float32)
    s = I.packing_batch([24, 60], tag=45)
    model = nb.Model(h, th32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 160, 64, shifts=True)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, 160, 64, train=True)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    teacher = I.init_params(h, seed=2).astype(np.float32).astype(np.float64)
    box64 = s.box.astype(np.float32).astype(np.float64)
    lab = O.energy_forces_virial(h, teacher, p32.astype(np.float64), s.types, box64, s.atom_off, pairs)
    E = torch.tensor(lab["Etot"], dtype=torch.float64, device="cuda")
    V = torch.tensor(lab["V"].reshape(-1, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(nb.NepError) as err:
        nb.param_grad(model, dsys, nl, ws, E, torch.tensor(np.ascontiguousarray(lab["F"].T), dtype=torch.float32,
                                                           device="cuda"), V)
    assert err.value.status == nb.NEP_ERR_UNSUPPORTED
    with pytest.raises(nb.NepError) as err:
        nb.autotune(model, dsys, nl, ws)
    assert err.value.status == nb.NEP_ERR_UNSUPPORTED
    ws64 = nb.Workspace64(model, s.n_atoms, s.n_cfg, train=True)
    F64 = torch.tensor(np.ascontiguousarray(lab["F"].T), dtype=torch.float64, device="cuda")
    g, loss = nb.param_grad_fp64(model, dsys, nl, ws64, E, F64, V)
    th = th32.astype(np.float64)
    idx = list(range(0, th.size, 37))
    ref = O.complex_step_grad(lambda t: O.loss_value(h, t, p32.astype(np.float64), s.types, box64, s.atom_off,
                                                     pairs, lab["Etot"], lab["F"], lab["V"]), th, idx)
    got = g.cpu().numpy()[idx]
    assert np.linalg.norm(got - ref) <= 1e-9 * max(np.linalg.norm(ref), 1e-30)

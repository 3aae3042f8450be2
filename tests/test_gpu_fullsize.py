"""Parity at the full workload sizes, in the launch configuration the bench
times, on sampled atoms the FP64 oracle evaluates one by one from their
neighbourhoods (oracle.evaluate_centers), plus properties that hold at any
size (zero net force, a symmetric virial, the FP64 total equal to the sum of
the per-atom energies).

* 900,000 atoms, 38-30-1 model, FP32: list with a 1 A skin and capacities
  160/80, ten velocity-Verlet steps captured in a CUDA graph (a rebuild at
  step 0), then a rebuild step; the forces of that step and the energies at
  its positions are sampled.
* 3,686,400 atoms, 52-64-1 model: FP32 at the FP32 bar and FP16 / BF16 at the
  mixed bar (force RMS <= 2 meV/A over the sample, energy <= 0.5 meV/atom).
* 1,024 replicas (N log-uniform in [64, 4096]), FP16 in one batched launch:
  four replicas checked whole against the oracle.
"""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_E, TOL_F = 1e-6, 1e-4
TOL_FRMS, TOL_E_ATOM = 2e-3, 5e-4
SKIN, DT, REBUILD = 1.0, 2.0, 10


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


def oracle_sample(h, th32, pos32, s, centers):
    pos32 = np.ascontiguousarray(pos32, np.float32)
    return O.evaluate_centers(h, th32.astype(np.float64), pos32, pos32.astype(np.float64), s.types,
                              s.box.astype(np.float32).astype(np.float64), s.atom_off, centers)


def test_md900k_sampled_after_graph_captured_steps(nb):
    import torch
    s, h = I.workload_md900k()
    N = s.n_atoms
    th32 = I.init_params(h).astype(np.float32)
    model = nb.Model(h, th32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(N, 160, 80, shifts=False)
    ws = nb.Workspace(model, N, 1, 160, 80)
    nb.neighbors(model, dsys, nl, SKIN, ws)
    e_atom, force, e_tot, vir = nb.energy_forces_virial(model, dsys, nl, ws)
    vel = torch.from_numpy(np.ascontiguousarray(I.maxwell_boltzmann(s.types, 900.0).astype(np.float32).T)).cuda()
    masses = I.MASSES.astype(np.float32)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for k in range(10):
            nb.md_step(model, dsys, nl, vel, force, e_tot, vir, masses, DT, SKIN, k % REBUILD == 0, ws,
                       stream=stream)
    g.replay()
    torch.cuda.synchronize()
    # a rebuild step leaves the positions wrapped into the box, as the oracle wants
    nb.md_step(model, dsys, nl, vel, force, e_tot, vir, masses, DT, SKIN, True, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    e2, f2, et2, v2 = nb.energy_forces_virial(model, dsys, nl, ws)
    assert torch.equal(f2, force)                       # same positions, same list: same bits
    pos32 = dsys.pos.cpu().numpy().T
    centers = np.random.default_rng(11).choice(N, 24, replace=False)
    ref = oracle_sample(h, th32, pos32, s, centers)
    E = e2.cpu().numpy()[ref["centers"]]
    F = f2.cpu().numpy().T[ref["centers"]]
    assert np.abs(E - ref["E"]).max() <= TOL_E
    assert np.abs(F - ref["F"]).max() <= TOL_F
    # any size: the FP64 total is the sum of the per-atom energies; the
    # forces of an isolated periodic system sum to zero; the virial of a
    # rotation-invariant energy is symmetric
    assert abs(float(et2[0]) - e2.double().sum().item()) <= 1e-6 * N
    fsum = f2.double().sum(1).abs().max().item()
    assert fsum <= 1e-7 * N                             # FP32 rounding of ~1e6 pair terms
    V = v2.cpu().numpy().reshape(3, 3)
    assert np.abs(V - V.T).max() <= 1e-6 * N


@pytest.fixture(scope="module")
def big_system():
    s, h = I.workload_mixed3m7()
    return s, h, I.init_params(h).astype(np.float32)


def test_mixed3m7_sampled(nb, big_system):
    s, h, th32 = big_system
    N = s.n_atoms
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(N, 80, 40, shifts=False)
    centers = np.random.default_rng(12).choice(N, 24, replace=False)
    ref = oracle_sample(h, th32, s.pos32(), s, centers)
    out = {}
    for prec in (0, 1, 2):
        model = nb.Model(h, th32, precision=prec)
        ws = nb.Workspace(model, N, 1, 80, 40)
        nb.neighbors(model, dsys, nl, 0.0, ws)
        assert nb.check_list(nl) == nb.NEP_OK
        e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
        out[prec] = (e.cpu().numpy()[ref["centers"]], f.cpu().numpy().T[ref["centers"]], float(et[0]))
        del ws, model
    E32, F32, Et32 = out[0]
    assert np.abs(E32 - ref["E"]).max() <= TOL_E
    assert np.abs(F32 - ref["F"]).max() <= TOL_F
    for prec in (1, 2):
        E, F, Et = out[prec]
        assert np.sqrt(np.mean((F - ref["F"]) ** 2)) <= TOL_FRMS
        assert np.abs(E - ref["E"]).mean() <= TOL_E_ATOM
        # total: the FP32 total is within 1e-6 eV/atom of FP64, so this bounds |dE|/N
        assert abs(Et - Et32) / N + 1e-6 <= TOL_E_ATOM


def test_replicas1024_sampled_whole(nb):
    s, h = I.workload_replicas1024()
    N, B = s.n_atoms, s.n_cfg
    th32 = I.init_params(h).astype(np.float32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(N, 160, 80, shifts=True)
    counts = np.diff(s.atom_off)
    picks = sorted({int(np.argmin(counts)), int(np.argmax(counts))}
                   | set(np.random.default_rng(13).choice(B, 2, replace=False).tolist()))
    res = {}
    for prec in (0, 1):
        model = nb.Model(h, th32, precision=prec)
        ws = nb.Workspace(model, N, B, 160, 80)
        nb.neighbors(model, dsys, nl, SKIN, ws)
        assert nb.check_list(nl) == nb.NEP_OK
        if prec:
            nb.autotune(model, dsys, nl, ws)             # as the bench runs it
        e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
        res[prec] = (e.cpu().numpy(), f.cpu().numpy().T, et.cpu().numpy())
        del ws, model
    p32 = s.pos32()
    for b in picks:
        a0, a1 = int(s.atom_off[b]), int(s.atom_off[b + 1])
        sb = I.System(pos=s.pos[a0:a1], types=s.types[a0:a1], box=s.box[b:b + 1],
                      atom_off=np.array([0, a1 - a0]))
        pairs = O.neighbor_pairs(p32[a0:a1], sb.box, sb.atom_off, h.rc_rad)
        ref = O.energy_forces_virial(h, th32.astype(np.float64), p32[a0:a1].astype(np.float64), sb.types,
                                     sb.box.astype(np.float32).astype(np.float64), sb.atom_off, pairs)
        e32, f32, et32 = res[0]
        assert np.abs(e32[a0:a1] - ref["E"]).max() <= TOL_E
        assert np.abs(f32[a0:a1] - ref["F"]).max() <= TOL_F
        assert abs(et32[b] - ref["Etot"][0]) <= 1e-6 * (a1 - a0)
        e16, f16, et16 = res[1]
        assert np.sqrt(np.mean((f16[a0:a1] - ref["F"]) ** 2)) <= TOL_FRMS
        assert abs(et16[b] - ref["Etot"][0]) / (a1 - a0) <= TOL_E_ATOM

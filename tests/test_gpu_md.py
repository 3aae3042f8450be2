"""The velocity-Verlet step (nep_md_step, through the C ABI) against the
FP64 oracle's integrator, and the energy conservation of a longer NVE run.

Tolerances, FP32 step against the FP64 oracle started from the same float32
positions, velocities and masses, over 12 steps of 2 fs with list rebuilds
(and wraps) at steps 0 and 10:
  positions   1e-4 A: each FP32 drift rounds x (ulp 2e-6 A at 25 A), and
              the FP32 forces (within 1e-6 eV/A of FP64 here) move the
              trajectory by less than that in 12 steps;
  velocities  1e-6 A/fs: a half kick changes v by dt/2 F/(m 103.6427), about
              1e-4 A/fs per eV/A, so FP32 force error and the position error
              above (through a force constant of order 10 eV/A^2) reach
              ~1e-7 A/fs in 12 steps.  A wrong unit factor, a species given
              another's mass or a missing half kick moves v by 1e-5 A/fs or
              more per step;
  forces      1e-4 eV/A (the parity bar);
  energies    1e-5 eV per atom: sum_i F_i . dx_i over the position error.
"""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_X, TOL_V, TOL_F, TOL_E = 1e-4, 1e-6, 1e-4, 1e-5
DT, SKIN = 2.0, 1.0


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


def start(nb, h, th32, s, cap, cap_ang):
    import torch
    model = nb.Model(h, th32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang, shifts=True)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, cap, cap_ang)
    nb.neighbors(model, dsys, nl, SKIN, ws)
    _, f, et, vir = nb.energy_forces_virial(model, dsys, nl, ws)
    v0 = I.maxwell_boltzmann(s.types, 900.0, atom_off=s.atom_off).astype(np.float32)
    vel = torch.from_numpy(np.ascontiguousarray(v0.T)).cuda()
    assert nb.check_list(nl) == nb.NEP_OK
    return model, dsys, nl, ws, f, et, vir, vel, v0


def test_md_step_matches_oracle_trajectory(nb):
    """Twelve steps of a three-configuration, three-species batch of uneven
    packings (64, 120 and 200 atoms; boxes below twice the list cutoff, so
    the list carries image shifts)."""
    h = I.HYPER_SMALL
    th32 = I.init_params(h).astype(np.float32)
    s = I.packing_batch([64, 120, 200], tag=91)
    m32 = I.MASSES.astype(np.float32)
    model, dsys, nl, ws, f, et, vir, vel, v0 = start(nb, h, th32, s, 160, 64)
    for k in range(12):
        nb.md_step(model, dsys, nl, vel, f, et, vir, m32, DT, SKIN, k % 10 == 0, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    x_g = dsys.pos.cpu().numpy().T.astype(np.float64)
    v_g = vel.cpu().numpy().T.astype(np.float64)
    f_g = f.cpu().numpy().T.astype(np.float64)
    e_g = et.cpu().numpy()

    box = s.box.astype(np.float32).astype(np.float64)
    r = O.velocity_verlet(h, th32.astype(np.float64), s.pos32().astype(np.float64), v0.astype(np.float64),
                          s.types, box, s.atom_off, m32.astype(np.float64), DT, 12)
    L = box[s.cfg_of_atom()]
    d = x_g - r["pos"]
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= TOL_X
    # both sides wrapped at step 10 and drifted once more: away from the box
    # faces the coordinates agree without any image shift
    far = np.all((r["pos"] > 0.05) & (r["pos"] < L - 0.05), axis=1)
    assert far.mean() > 0.9 and np.abs(x_g[far] - r["pos"][far]).max() <= TOL_X
    assert np.abs(v_g - r["vel"]).max() <= TOL_V
    assert np.abs(f_g - r["F"]).max() <= TOL_F
    Nb = np.diff(s.atom_off)
    assert np.all(np.abs(e_g - r["epot"][-1]) <= TOL_E * Nb)
    # momentum stays at its start value per configuration (sum F = 0)
    for b in range(s.n_cfg):
        sl = slice(s.atom_off[b], s.atom_off[b + 1])
        p = (m32[s.types[sl]][:, None] * v_g[sl]).sum(0)
        assert np.abs(p).max() < 1e-4


def test_nve_energy_conservation_216(nb):
    """300 steps (600 fs) of the 216-atom cell at 900 K: the total energy
    (FP64 energy sum from the GPU, kinetic energy from its velocities)
    stays within 1e-4 eV per atom of its start; over the first 30 steps it
    follows the oracle's FP64 run within 1e-5 eV per atom."""
    h = I.HYPER_SMALL
    th32 = I.init_params(h).astype(np.float32)
    s, _ = I.workload_cell216()
    m32 = I.MASSES.astype(np.float32)
    model, dsys, nl, ws, f, et, vir, vel, v0 = start(nb, h, th32, s, 112, 56)
    ke = lambda v: O.kinetic_energy(v, s.types, m32.astype(np.float64), s.atom_off)[0]
    e0 = et.item() + ke(v0.astype(np.float64))
    tot = []
    for k in range(300):
        nb.md_step(model, dsys, nl, vel, f, et, vir, m32, DT, SKIN, k % 10 == 0, ws)
        tot.append(et.item() + ke(vel.cpu().numpy().T.astype(np.float64)))
    assert nb.check_list(nl) == nb.NEP_OK
    tot = np.array(tot)
    N = s.n_atoms
    assert np.abs(tot - e0).max() / N <= 1e-4
    r = O.velocity_verlet(h, th32.astype(np.float64), s.pos32().astype(np.float64), v0.astype(np.float64),
                          s.types, s.box.astype(np.float32).astype(np.float64), s.atom_off,
                          m32.astype(np.float64), DT, 30)
    ref = r["epot"][:, 0] + r["ekin"][:, 0]
    assert np.abs(tot[:30] - ref).max() / N <= TOL_E

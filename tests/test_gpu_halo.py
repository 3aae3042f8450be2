"""The point-to-point slab decomposition on the GPU (halo.py through
libnep), with the ranks run one after another in one process (run_emulated:
no kernel of one rank waits on another's).

  * The forces of every rank's own atoms at the start, gathered by atom id,
    against the FP64 oracle on sampled atoms (the parity bar, 1e-4 eV/A and
    1e-6 eV per atom for the energy sum) and against the whole-system call.
  * Twelve velocity-Verlet steps (a rebuild with migration at step 10)
    against nep_md_step on the whole system: positions 1e-4 A, velocities
    1e-5 A/fs, energy 1e-5 eV per atom (FP32 sums in another order and
    positions in a shifted frame differ by a few ulps per step)."""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SKIN = 1.0


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


def ranks_for(nb, model, s, v, world):
    from paper_2607_06969_gb300 import halo as HL
    L = s.box[0]
    slabs, halo = HL.plan(float(L[0]), world, model.h.rc_rad, SKIN)
    ops = HL.LibOps(model)
    ranks = []
    for r, (lo, hi) in enumerate(slabs):
        k = HL.SlabRank(ops, r, world, L, lo, hi, halo, SKIN, I.MASSES, dt=2.0, rebuild_every=10, cap=112,
                        cap_ang=56, rc=model.h.rc_rad)
        k.load(s.pos32(), s.types, v)
        ranks.append(k)
    return ranks


def gather(ranks, N, field):
    out = np.full((N, 3), np.nan)
    for k in ranks:
        out[k.gid[0].cpu().numpy()] = getattr(k, field).T.cpu().numpy()
    assert not np.isnan(out).any()
    return out


@pytest.mark.parametrize("world", [2, 4])
def test_start_forces_against_oracle_and_whole_system(nb, world):
    import torch
    from paper_2607_06969_gb300 import halo as HL
    h = I.HYPER_SMALL
    th32 = I.init_params(h).astype(np.float32)
    s = I.rocksalt(14, vacancy=0.2, tag=31)
    v = I.maxwell_boltzmann(s.types, 900.0).astype(np.float32)
    model = nb.Model(h, th32)
    ranks = ranks_for(nb, model, s, v, world)
    HL.run_emulated([k.start() for k in ranks])
    for k in ranks:
        k.check()
    F = gather(ranks, s.n_atoms, "force")
    e, vir = HL.totals(ranks)
    # whole system
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 112, 56, shifts=False)
    ws = nb.Workspace(model, s.n_atoms, 1, 112, 56)
    nb.neighbors(model, dsys, nl, SKIN, ws)
    _, fw, ew, vw = nb.energy_forces_virial(model, dsys, nl, ws)
    assert np.abs(F - fw.cpu().numpy().T).max() <= 1e-5
    assert abs(e.item() - ew.item()) <= 1e-6 * s.n_atoms
    assert (vir - vw.cpu()).abs().max().item() <= 1e-6 * s.n_atoms
    # oracle on atoms next to the slab faces and inside the slabs
    p32 = s.pos32()
    L = float(s.box[0, 0])
    faces = np.array([L * r / world for r in range(world + 1)])
    dface = np.abs(p32[:, 0].astype(np.float64)[:, None] - faces[None, :]).min(1)
    rng = np.random.default_rng(31)
    c = np.concatenate([rng.choice(np.nonzero(dface < 1.0)[0], 40, replace=False),
                        rng.choice(np.nonzero(dface >= 1.0)[0], 16, replace=False)])
    ref = O.evaluate_centers(h, th32.astype(np.float64), p32, p32.astype(np.float64), s.types,
                             s.box.astype(np.float32).astype(np.float64), s.atom_off, c)
    assert np.abs(F[ref["centers"]] - ref["F"]).max() <= 1e-4


@pytest.mark.parametrize("world", [2, 3])
def test_halo_md_tracks_whole_system_md(nb, world):
    import torch
    from paper_2607_06969_gb300 import halo as HL
    h = I.HYPER_SMALL
    s = I.rocksalt(14, vacancy=0.2, tag=32)
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    masses = I.MASSES.astype(np.float32)
    v0 = I.maxwell_boltzmann(s.types, 900.0).astype(np.float32)
    # whole system
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 112, 56, shifts=False)
    ws = nb.Workspace(model, s.n_atoms, 1, 112, 56)
    nb.neighbors(model, dsys, nl, SKIN, ws)
    _, force, et, vir = nb.energy_forces_virial(model, dsys, nl, ws)
    vel = torch.from_numpy(np.ascontiguousarray(v0.T)).cuda()
    for k in range(1, 13):
        nb.md_step(model, dsys, nl, vel, force, et, vir, masses, 2.0, SKIN, k % 10 == 0, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    # the decomposition
    ranks = ranks_for(nb, model, s, v0, world)
    HL.run_emulated([k.start() for k in ranks])
    for _ in range(12):
        HL.run_emulated([k.step() for k in ranks])
    for k in ranks:
        k.check()
    pos = gather(ranks, s.n_atoms, "pos")
    vv = gather(ranks, s.n_atoms, "vel")
    L = s.box[0]
    d = pos - dsys.pos.cpu().numpy().T
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 1e-4
    assert np.abs(vv - vel.cpu().numpy().T).max() <= 1e-5
    e, _ = HL.totals(ranks)
    assert abs(e.item() - et.item()) <= 1e-5 * s.n_atoms
    for k in ranks:                     # after the migration at step 10 every atom is near its own slab
        x = k.pos[0].cpu().numpy()
        assert np.all((x > k.lo - 1.0) & (x < k.hi + 1.0))

"""The point-to-point slab decomposition with two real processes, both on
cuda:0, exchanging their halos over gloo through host memory (no kernel of
one rank waits on the other): twelve velocity-Verlet steps with a rebuild
and migration at step 10, gathered by atom id and compared with the
single-process nep_md_step trajectory within the FP32 ordering bar
(positions 1e-4 A, velocities 1e-5 A/fs, energy 1e-5 eV per atom)."""
import os
import socket

import numpy as np
import pytest

from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SKIN, STEPS = 1.0, 12


def _system():
    return I.rocksalt(14, vacancy=0.2, tag=6), I.HYPER_SMALL


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from paper_2607_06969_gb300 import binding as nb
    from paper_2607_06969_gb300 import halo as HL
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    s, h = _system()
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    v0 = I.maxwell_boltzmann(s.types, 900.0).astype(np.float32)
    slabs, halo = HL.plan(float(s.box[0, 0]), world, h.rc_rad, SKIN)
    lo, hi = slabs[rank]
    k = HL.SlabRank(HL.LibOps(model), rank, world, s.box[0], lo, hi, halo, SKIN, I.MASSES, dt=2.0,
                    rebuild_every=10, cap=112, cap_ang=56, rc=h.rc_rad)
    k.load(s.pos32(), s.types, v0)
    HL.run_dist(k.start(), dist, rank, world, host_staging=True)
    for _ in range(STEPS):
        HL.run_dist(k.step(), dist, rank, world, host_staging=True)
    e, _ = HL.totals(k, dist)
    torch.cuda.synchronize()
    q.put((rank, k.gid[0].cpu().numpy(), k.pos.T.cpu().numpy(), k.vel.T.cpu().numpy(), float(e.item()),
           nb.check_list(k.nl)))
    dist.destroy_process_group()


def test_two_process_halo_md():
    import torch
    import torch.multiprocessing as mp
    from paper_2607_06969_gb300 import build as B
    from paper_2607_06969_gb300 import binding as nb
    B.build()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=600) for _ in ps), key=lambda x: x[0])
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    s, h = _system()
    pos = np.full((s.n_atoms, 3), np.nan)
    vel = np.full((s.n_atoms, 3), np.nan)
    for _, g, p_, v_, e, st in res:
        assert st == nb.NEP_OK
        assert np.all(np.isnan(pos[g, 0]))           # every atom owned by one rank
        pos[g], vel[g] = p_, v_
    assert not np.isnan(pos).any()
    assert res[0][4] == res[1][4]                   # the all-reduced energy, on both ranks
    # the single-process trajectory
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 112, 56, shifts=False)
    ws = nb.Workspace(model, s.n_atoms, 1, 112, 56)
    nb.neighbors(model, dsys, nl, SKIN, ws)
    _, force, et, vir = nb.energy_forces_virial(model, dsys, nl, ws)
    v = torch.from_numpy(np.ascontiguousarray(I.maxwell_boltzmann(s.types, 900.0).astype(np.float32).T)).cuda()
    for k in range(1, STEPS + 1):
        nb.md_step(model, dsys, nl, v, force, et, vir, I.MASSES.astype(np.float32), 2.0, SKIN, k % 10 == 0, ws)
    torch.cuda.synchronize()
    L = s.box[0]
    d = pos - dsys.pos.cpu().numpy().T
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 1e-4
    assert np.abs(vel - v.cpu().numpy().T).max() <= 1e-5
    assert abs(res[0][4] - et.item()) <= 1e-5 * s.n_atoms

"""The slab decomposition with two real processes (gloo all-reduce through
host memory, both on cuda:0; no kernel of one rank waits on the other):
twelve velocity-Verlet steps, the replicated state identical on both ranks
(the combined forces are exact sums of disjoint rows), and equal to the
single-process nep_md_step trajectory within the FP32 ordering bar."""
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
    from paper_2607_06969_gb300 import spatial as SP
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    s, h = _system()
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    gsys = nb.DeviceSystem.from_inputs(s)
    vel = torch.from_numpy(np.ascontiguousarray(I.maxwell_boltzmann(s.types, 900.0).astype(np.float32).T)).cuda()
    slabs, halo = SP.plan_slabs(float(s.box[0, 0]), world, h.rc_rad, SKIN)
    lo, hi = slabs[rank]
    dom = SP.SlabDomain(model, gsys, lo, hi, halo, SKIN, 112, 56)
    md = SP.SpatialMD(model, gsys, vel, I.MASSES.astype(np.float32), [dom],
                      reduce=lambda f, e, v: SP.combine_owned(dist, f, e, v), dt=2.0, skin=SKIN, rebuild_every=10)
    md.start()
    for _ in range(STEPS):
        md.step()
    torch.cuda.synchronize()
    q.put((rank, gsys.pos.cpu().numpy(), vel.cpu().numpy(), float(md.e_tot.item()), nb.check_list(dom.nl)))
    dist.destroy_process_group()


def test_two_process_slab_md():
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
    (_, pos0, vel0, e0, st0), (_, pos1, vel1, e1, st1) = res
    assert st0 == nb.NEP_OK and st1 == nb.NEP_OK
    assert np.array_equal(pos0, pos1) and np.array_equal(vel0, vel1) and e0 == e1
    # the single-process trajectory
    s, h = _system()
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 112, 56, shifts=False)
    ws = nb.Workspace(model, s.n_atoms, 1, 112, 56)
    nb.neighbors(model, dsys, nl, SKIN, ws)
    _, force, et, vir = nb.energy_forces_virial(model, dsys, nl, ws)
    vel = torch.from_numpy(np.ascontiguousarray(I.maxwell_boltzmann(s.types, 900.0).astype(np.float32).T)).cuda()
    for k in range(1, STEPS + 1):
        nb.md_step(model, dsys, nl, vel, force, et, vir, I.MASSES.astype(np.float32), 2.0, SKIN, k % 10 == 0, ws)
    torch.cuda.synchronize()
    assert np.abs(pos0 - dsys.pos.cpu().numpy()).max() <= 1e-4
    assert np.abs(vel0 - vel.cpu().numpy()).max() <= 1e-5
    assert abs(e0 - et.item()) <= 1e-5 * s.n_atoms

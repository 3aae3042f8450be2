"""The point-to-point slab decomposition (halo.py) on the CPU: migration of
atoms between slabs, the ghost bands of each face, the periodic images of the
end slabs and the exchange pattern, checked against a whole-system run.

The library's kernels need a GPU, so these tests drive SlabRank with a
stand-in for its device operations (torch on the CPU: the same band, take,
place and kick semantics as nep.h states them, and a short-ranged pair
potential in place of the NEP evaluation).  The decomposition's bookkeeping
is what is under test; the NEP evaluation through the same code is tested
on the GPU (test_gpu_halo.py).  The ranks run in one process in lockstep
(run_emulated) and as world_size-2 and 3 gloo process groups (run_dist)."""
import os
import socket

import numpy as np
import pytest
import torch

from paper_2607_06969_gb300 import halo as HL
from paper_2607_06969_gb300 import inputs as I

RC, SKIN, EPS, DT = 3.0, 0.5, 0.5, 2.0
MASSES = I.MASSES
KAPPA = 103.6427


def pair_forces(pos, L_periodic, n_owned, periodic_x):
    """phi(r) = EPS (1 - r/RC)^3 for r < RC.  Forces on the first n_owned
    rows from every row; energy of those rows (half of each pair's phi)."""
    d = pos[None, :, :] - pos[:n_owned, None, :]              # r_j - r_i
    for a in range(3):
        if a > 0 or periodic_x:
            d[..., a] -= L_periodic[a] * torch.round(d[..., a] / L_periodic[a])
    r = torch.sqrt((d * d).sum(-1))
    mask = (r < RC) & (r > 0)
    rs = torch.where(mask, r, torch.ones_like(r))
    dphi = torch.where(mask, -3.0 * EPS / RC * (1 - rs / RC) ** 2, torch.zeros_like(r))
    F = (dphi / rs)[..., None] * d * mask[..., None]            # F_i = sum_j phi'(r) r_ij / r
    F = F.sum(1)
    e = torch.where(mask, 0.5 * EPS * (1 - rs / RC) ** 3, torch.zeros_like(r)).sum()
    return F, e


class StandInOps:
    """CPU stand-in for halo.LibOps (test infrastructure only)."""
    device = "cpu"
    torch = torch

    def empty(self, shape, dtype):
        return torch.empty(shape, dtype=dtype)

    def band(self, pos, n, lo, hi):
        x = pos[0, :n]
        return torch.nonzero((x >= lo) & (x < hi)).reshape(-1).to(torch.int32)

    def take(self, src, n_src, idx):
        return src[:, :n_src][:, idx.long()].contiguous()

    def place(self, src, n, box_x, x_center, x_origin, dst, stride, offset):
        flat = dst.reshape(-1)
        for c in range(src.shape[0]):
            v = src[c, :n].clone()
            if c == 0 and box_x > 0:
                v = (v - box_x * torch.round((v - x_center) / box_x)) - x_origin
            flat[c * stride + offset:c * stride + offset + n] = v

    def kick(self, sys_, vel, force, masses, half_dt, drift_dt):
        n = sys_.n_atoms
        if n == 0:
            return
        t = sys_.type[:n].long()
        inv = torch.tensor(1.0 / (np.asarray(masses, np.float64) * KAPPA), dtype=torch.float32)[t]
        vel[:, :n] += half_dt * force[:, :n] * inv[None, :]
        if drift_dt > 0:
            sys_.pos[:, :n] += drift_dt * vel[:, :n]

    def wrap(self, sys_):
        n = sys_.n_atoms
        L = torch.tensor(sys_.box_host[0], dtype=torch.float32)[:, None]
        sys_.pos[:, :n] -= L * torch.floor(sys_.pos[:, :n] / L)

    def neighbors(self, loc, nl, skin, ws):
        pass

    def evaluate_owned(self, loc, nl, n_owned, force, e_tot, vir, ws):
        n = loc.n_atoms
        pos = loc.pos[:, :n].T.double()
        F, e = pair_forces(pos, torch.tensor(loc.box_host[0], dtype=torch.float64), n_owned, periodic_x=False)
        force[:, :n] = 0
        force[:, :n_owned] = F.T.float()
        e_tot[0] = e

    def workspace(self, n_atoms, cap, cap_ang):
        return None

    def check_list(self, nl):
        pass


def reference(pos, vel, types, L, steps):
    """The whole system in FP64 with the same stand-in potential."""
    pos = torch.tensor(pos, dtype=torch.float64)
    vel = torch.tensor(vel, dtype=torch.float64)
    Lt = torch.tensor(L, dtype=torch.float64)
    inv = torch.tensor(1.0 / (MASSES[types] * KAPPA))[:, None]
    F, _ = pair_forces(pos, Lt, pos.shape[0], periodic_x=True)
    for _ in range(steps):
        vel = vel + 0.5 * DT * F * inv
        pos = pos + DT * vel
        F, _ = pair_forces(pos, Lt, pos.shape[0], periodic_x=True)
        vel = vel + 0.5 * DT * F * inv
    return pos.numpy(), vel.numpy()


def workload(seed=0):
    s = I.packing_batch([600], tag=60 + seed)
    v = 4.0 * I.maxwell_boltzmann(s.types, 900.0, atom_off=s.atom_off)   # hot: atoms cross faces
    return s, v


def make_ranks(s, v, world):
    L = s.box[0]
    slabs, halo = HL.plan(float(L[0]), world, RC, SKIN)
    ranks = []
    for r, (lo, hi) in enumerate(slabs):
        k = HL.SlabRank(StandInOps(), r, world, L, lo, hi, halo, SKIN, MASSES, dt=DT, rebuild_every=5,
                        cap=64, cap_ang=32, rc=RC)
        k.load(s.pos32(), s.types, v.astype(np.float32))
        ranks.append(k)
    return ranks


def collect(ranks, N):
    pos = np.full((N, 3), np.nan)
    vel = np.full((N, 3), np.nan)
    for k in ranks:
        g = k.gid[0].numpy()
        assert np.all(np.isnan(pos[g, 0]))                 # every atom owned once
        pos[g] = k.pos.T.numpy()
        vel[g] = k.vel.T.numpy()
    assert not np.isnan(pos).any()
    return pos, vel


def compare(pos, vel, s, v, steps):
    L = s.box[0]
    ref_p, ref_v = reference(s.pos32().astype(np.float64), v.astype(np.float32).astype(np.float64), s.types, L,
                             steps)
    d = pos - ref_p
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 2e-4
    assert np.abs(vel - ref_v).max() < 2e-5


def test_plan_rejects_narrow_slabs_and_one_rank():
    with pytest.raises(ValueError):
        HL.plan(30.0, 1, 7.0, 1.0)
    with pytest.raises(ValueError):
        HL.plan(30.0, 2, 7.0, 1.0)          # 15 A slabs, 16 A halo
    slabs, halo = HL.plan(300.0, 8, 7.0, 1.0)
    assert halo == 16.0 and slabs[0] == (0.0, 37.5) and slabs[-1][1] == 300.0


@pytest.mark.parametrize("world", [2, 3])
def test_emulated_ranks_track_the_whole_system(world):
    s, v = workload()
    ranks = make_ranks(s, v, world)
    HL.run_emulated([k.start() for k in ranks])
    steps = 17                                      # rebuilds (and migrations) at steps 5, 10 and 15
    moved = 0
    for _ in range(steps):
        before = [set(k.gid[0].tolist()) for k in ranks]
        HL.run_emulated([k.step() for k in ranks])
        moved += sum(len(b - set(k.gid[0].tolist())) for b, k in zip(before, ranks))
    assert moved > 0                                # atoms did change slabs
    pos, vel = collect(ranks, s.n_atoms)
    compare(pos, vel, s, v, steps)
    for k in ranks:                                 # own atoms inside their slab after the last rebuild
        x = k.pos[0].numpy()
        assert np.all((x > k.lo - 1.0) & (x < k.hi + 1.0))


def _free_port():
    with socket.socket() as k:
        k.bind(("127.0.0.1", 0))
        return k.getsockname()[1]


def _worker(rank, world, port, steps, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, v = workload()
        k = make_ranks(s, v, world)[rank]
        HL.run_dist(k.start(), dist, rank, world)
        for _ in range(steps):
            HL.run_dist(k.step(), dist, rank, world)
        q.put((rank, k.gid[0].numpy(), k.pos.T.numpy(), k.vel.T.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_track_the_whole_system(world):
    import torch.multiprocessing as mp
    steps = 12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s, v = workload()
    pos = np.full((s.n_atoms, 3), np.nan)
    vel = np.full((s.n_atoms, 3), np.nan)
    for _, g, p_, v_ in out:
        assert np.all(np.isnan(pos[g, 0]))
        pos[g], vel[g] = p_, v_
    assert not np.isnan(pos).any()
    compare(pos, vel, s, v, steps)

"""Data parallelism over configurations: shard bounds, the weighted gradient
all-reduce over a world_size-2 gloo group on the CPU, and (GPU) the shard
gradients of nep_param_grad recombining into the full-batch gradient."""
import os
import socket

import numpy as np
import pytest

from paper_2607_06969_gb300 import dp
from paper_2607_06969_gb300 import inputs as I


def test_shard_bounds_cover_and_balance():
    rng = np.random.default_rng(3)
    counts = rng.integers(24, 513, size=128)
    off = np.concatenate([[0], np.cumsum(counts)])
    for world in (1, 2, 3, 4, 8, 128):
        b = dp.shard_bounds(off, world)
        assert len(b) == world and b[0][0] == 0 and b[-1][1] == 128
        assert all(b0 < b1 for b0, b1 in b)                          # one config at least
        assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))  # contiguous, no overlap
        atoms = [off[b1] - off[b0] for b0, b1 in b]
        if world <= 8:                                                # within one config of fair
            assert max(atoms) - off[-1] / world <= counts.max()
    with pytest.raises(ValueError):
        dp.shard_bounds(off, 129)


def test_replica_batch_shards_by_atoms():
    """The 1,024-replica batch (N log-uniform in [64, 4096]) split over 2-8
    ranks: every rank within one replica of an equal share of the atoms."""
    counts = np.asarray(I.loguniform_counts(1024, 64, 4096, tag=4))
    off = np.concatenate([[0], np.cumsum(counts)])
    for world in (2, 4, 8):
        b = dp.shard_bounds(off, world)
        atoms = np.array([off[b1] - off[b0] for b0, b1 in b])
        assert atoms.sum() == off[-1]
        assert np.all(np.abs(atoms - off[-1] / world) <= counts.max())


def test_shard_system_round_trip():
    s = I.packing_batch([24, 31, 57, 100], tag=95)
    sub = dp.shard_system(s, 1, 3)
    assert sub.n_cfg == 2 and sub.n_atoms == 31 + 57
    assert np.array_equal(sub.atom_off, [0, 31, 88])
    assert np.array_equal(sub.pos, s.pos[24:112]) and np.array_equal(sub.types, s.types[24:112])


def _free_port():
    with socket.socket() as k:
        k.bind(("127.0.0.1", 0))
        return k.getsockname()[1]


def _worker(rank, world, port, off, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B = len(off) - 1
        b0, b1 = dp.shard_bounds(off, world)[rank]
        # a per-configuration gradient and loss known on every rank: g_b[k] = sin(b + k/7)
        k = np.arange(50)
        g_b = np.array([np.sin(b + k / 7.0) for b in range(B)])
        l_b = np.arange(B, dtype=np.float64) ** 2
        grad = torch.tensor(g_b[b0:b1].mean(0), dtype=torch.float32)    # what nep_param_grad returns
        loss = torch.tensor([l_b[b0:b1].mean()], dtype=torch.float64)
        dp.allreduce_mean(dist, grad, loss, b1 - b0, B)
        q.put((rank, grad.numpy().astype(np.float64), float(loss[0]), g_b.mean(0), l_b.mean()))
    finally:
        dist.destroy_process_group()


def test_gloo_weighted_allreduce_world2():
    import torch.multiprocessing as mp
    off = np.array([0, 24, 31 + 24, 31 + 24 + 400, 31 + 24 + 400 + 57, 31 + 24 + 400 + 57 + 100])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, off, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, g, l, g_ref, l_ref in out:
        assert np.allclose(g, g_ref, atol=2e-7)        # the full-batch mean, on every rank
        assert l == pytest.approx(l_ref, rel=1e-12)
    assert np.array_equal(out[0][1], out[1][1])        # identical replicas


@pytest.mark.gpu
def test_shard_gradients_recombine_on_gpu():
    import torch
    from oracle import nep_oracle as O
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding as nb
    h = I.HYPER_SMALL
    s = I.packing_batch([24, 40, 57, 33, 90], tag=96)
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    teacher = I.init_params(h, seed=I.SEED_TEACHER).astype(np.float32).astype(np.float64)
    lab = O.energy_forces_virial(h, teacher, p32.astype(np.float64), s.types,
                                 s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)
    model = nb.Model(h, I.init_params(h).astype(np.float32))

    def grad_of(b0, b1):
        sub = dp.shard_system(s, b0, b1)
        a0, a1 = s.atom_off[b0], s.atom_off[b1]
        d = nb.DeviceSystem.from_inputs(sub)
        nl = nb.NeighborList(sub.n_atoms, 112, 56)
        ws = nb.Workspace(model, sub.n_atoms, sub.n_cfg, 112, 56, train=True)
        nb.neighbors(model, d, nl, 0.0, ws)
        E = torch.tensor(lab["Etot"][b0:b1], dtype=torch.float64, device="cuda")
        F = torch.tensor(np.ascontiguousarray(lab["F"][a0:a1].T), dtype=torch.float32, device="cuda")
        V = torch.tensor(lab["V"].reshape(-1, 9)[b0:b1], dtype=torch.float64, device="cuda")
        g, l = nb.param_grad(model, d, nl, ws, E, F, V)
        assert nb.check_list(nl) == nb.NEP_OK
        return g.cpu().numpy().astype(np.float64), float(l.item())

    full_g, full_l = grad_of(0, s.n_cfg)
    for world in (2, 3):
        g = np.zeros_like(full_g)
        l = 0.0
        for b0, b1 in dp.shard_bounds(s.atom_off, world):
            gr, lr = grad_of(b0, b1)
            g += (b1 - b0) / s.n_cfg * gr
            l += (b1 - b0) / s.n_cfg * lr
        assert np.linalg.norm(g - full_g) <= 1e-5 * np.linalg.norm(full_g)
        assert l == pytest.approx(full_l, rel=1e-6)

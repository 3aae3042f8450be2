"""Host logic of the spatial decomposition: slab planning, and the
all-reduce that combines the ranks' owned rows (gloo, world size 2, CPU)."""
import os

import numpy as np
import pytest

from paper_2607_06969_gb300 import spatial as SP


def test_plan_slabs_cover_and_reject_overlapping_halos():
    slabs, halo = SP.plan_slabs(300.0, 4, 7.0, 1.0)
    assert halo == 16.0
    assert slabs[0][0] == 0.0 and slabs[-1][1] == 300.0
    assert all(a[1] == b[0] for a, b in zip(slabs, slabs[1:]))
    assert SP.plan_slabs(84.0, 1, 7.0, 1.0)[0] == [(0.0, 84.0)]
    with pytest.raises(ValueError):
        SP.plan_slabs(60.0, 2, 7.0, 1.0)          # 30 + 2 * 16 > 60


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = 10
    full = torch.arange(3 * N, dtype=torch.float32).reshape(3, N) + 0.5
    owned = [np.arange(0, 4), np.arange(4, N)][rank]
    f = torch.zeros(3, N)
    f[:, owned] = full[:, owned]
    e = torch.tensor([1.5 + rank], dtype=torch.float64)
    v = torch.full((1, 9), 0.25 * (rank + 1), dtype=torch.float64)
    SP.combine_owned(dist, f, e, v)
    out.put((rank, torch.equal(f, full), e.item(), v[0, 0].item()))
    dist.destroy_process_group()


def test_combine_owned_gloo_world2():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, same, e, v in res:
        assert same and e == 4.0 and v == 0.75

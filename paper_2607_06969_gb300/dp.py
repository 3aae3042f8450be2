"""Data-parallel training over configurations (one process per GPU).

The batch loss is a mean over configurations, L = 1/B sum_b L_b (loss
modes 0 and 1 of nep_param_grad), so its gradient is the mean of the
per-configuration gradients.  Each rank takes a contiguous shard of B_r
configurations, nep_param_grad returns the mean over its shard, and

    grad = sum_r (B_r / B) grad_r,    L = sum_r (B_r / B) L_r

is one all-reduce (sum) of the P-float gradient and the loss after each rank
scales its own share.  Every rank then applies the same Adam step to the same
parameters, so the replicas stay identical without a parameter broadcast.

Shards are balanced by atom count (the gradient cost is per atom), keep the
configuration order, and give every rank at least one configuration.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(atom_off, world: int) -> list[tuple[int, int]]:
    """Contiguous configuration ranges [b0, b1) per rank, balanced by atoms.
    Rank r ends at the first configuration boundary at or beyond r+1 equal
    atom shares, with at least one configuration per rank."""
    atom_off = np.asarray(atom_off, np.int64)
    B = atom_off.size - 1
    if world < 1 or world > B:
        raise ValueError(f"need 1 <= world ({world}) <= number of configurations ({B})")
    N = int(atom_off[-1])
    bounds, b0 = [], 0
    for r in range(world):
        if r == world - 1:
            b1 = B
        else:
            target = N * (r + 1) / world
            b1 = int(np.searchsorted(atom_off, target, side="left"))
            b1 = max(b1, b0 + 1)                   # at least one configuration here
            b1 = min(b1, B - (world - 1 - r))      # and one for each later rank
        bounds.append((b0, b1))
        b0 = b1
    return bounds


def shard_system(s, b0: int, b1: int):
    """The configurations [b0, b1) of an inputs.System as a System of their own."""
    from .inputs import System
    a0, a1 = int(s.atom_off[b0]), int(s.atom_off[b1])
    return System(pos=s.pos[a0:a1], types=s.types[a0:a1], box=s.box[b0:b1],
                  atom_off=np.asarray(s.atom_off[b0:b1 + 1]) - a0)


def allreduce_mean(dist, grad, loss, n_local: int, n_total: int) -> None:
    """In place: grad <- sum_r (n_r/n) grad_r and loss <- sum_r (n_r/n) loss_r
    over the process group (torch tensors on the rank's device)."""
    w = n_local / n_total
    grad.mul_(w)
    dist.all_reduce(grad)
    if loss is not None:
        loss.mul_(w)
        dist.all_reduce(loss)

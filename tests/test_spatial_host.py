"""Host logic of the spatial decomposition: slab planning, a slab's local
frame, and, with the FP64 oracle, the reason for the two-layer halo: a slab's local system of
owned atoms and ghosts within 2 rc reproduces every owned atom's energy,
force and per-atom virial (so the owned sums add up to the whole system's
E and V), and one layer does not."""

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



def _slab_local(pos, L, lo, hi, halo):
    """Owned atoms (x in [lo, hi)) then ghosts (the first image k = -1, 0, 1
    whose x lies within `halo` of the slab), each in atom order, and their
    positions in the slab's frame (x - (lo - halo))."""
    owned, ghosts, img = [], [], []
    for i, x in enumerate(pos[:, 0]):
        if lo <= x < hi:
            owned.append(i)
            continue
        for k in (-1, 0, 1):
            xs = x + k * L[0]
            if lo - halo <= xs < lo or hi <= xs < hi + halo:
                ghosts.append(i)
                img.append(k)
                break
    idx = np.array(owned + ghosts, dtype=np.int64)
    lp = pos[idx].copy()
    lp[:, 0] += np.array([0] * len(owned) + img) * L[0] - (lo - halo)
    return idx, len(owned), lp


def _oracle_efv(h, th, pos, types, box, rc):
    from oracle import nep_oracle as O
    off = np.array([0, len(types)])
    pr = O.neighbor_pairs(pos.astype(np.float32), box, off, rc)
    return O.energy_forces_virial(h, th, pos, types, box, off, pr)


def test_two_layer_halo_reproduces_owned_atoms_in_the_oracle():
    from paper_2607_06969_gb300 import inputs as I
    h = I.Hyper(n_types=3, n_rad=3, n_ang=2, k_rad=4, k_ang=3, l_max=4, has_4body=1, n_hidden=4,
                rc_rad=5.0, rc_ang=4.0)
    th = I.init_params(h, seed=31)
    rng = np.random.default_rng(12)
    g = np.stack(np.meshgrid(np.arange(15), np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    pos = 3.0 * g + 1.5 + rng.normal(0.0, 0.2, size=g.shape)
    types = rng.integers(0, 3, size=len(pos)).astype(np.int32)
    L = np.array([45.0, 12.0, 12.0])
    whole = _oracle_efv(h, th, pos, types, L[None, :], h.rc_rad)
    from oracle import nep_oracle as O
    slabs, _ = SP.plan_slabs(L[0], 2, h.rc_rad, 0.0)
    e_sum, v_sum = 0.0, np.zeros((3, 3))
    for halo, exact in ((2.0 * h.rc_rad, True), (h.rc_rad, False)):
        worst = 0.0
        for lo, hi in slabs:
            idx, n_own, lp = _slab_local(pos, L, lo, hi, halo)
            box = np.array([[hi - lo + 2.0 * halo + h.rc_rad + 1.0, L[1], L[2]]])
            loc = _oracle_efv(h, th, lp, types[idx], box, h.rc_rad)
            own = idx[:n_own]
            worst = max(worst, np.abs(loc["F"][:n_own] - whole["F"][own]).max())
            if exact:
                assert np.allclose(loc["E"][:n_own], whole["E"][own], rtol=0, atol=1e-11)
                e_sum += loc["E"][:n_own].sum()
                # per-atom virials W_i = -sum_j f_ij (x) r_ij of the owned atoms
                c = O.evaluate_centers(h, th, lp.astype(np.float32), lp, types[idx], box,
                                       np.array([0, len(idx)]), np.arange(n_own))
                v_sum += c["W"].sum(0)
        if exact:
            assert worst < 1e-10
            assert abs(e_sum - whole["Etot"][0]) < 1e-10
            assert np.allclose(v_sum, whole["V"][0], rtol=0, atol=1e-9)
        else:
            assert worst > 1e-6            # ghosts' own neighbourhoods cut short


def test_slab_domain_frame_and_capacity():
    """A slab's local frame: origin lo - halo, a local box whose x exceeds
    slab + 2 halo by more than rc + skin (no local image in range), and a
    local capacity that covers the slab's share of the atoms."""
    from types import SimpleNamespace

    import torch
    h = SimpleNamespace(rc_rad=7.0)
    model = SimpleNamespace(h=h)
    N, L = 900_000, np.array([[300.0, 300.0, 300.0]], np.float32)
    g = SimpleNamespace(n_cfg=1, n_atoms=N, box_host=L, pos=torch.zeros(3, 1))
    slabs, halo = SP.plan_slabs(300.0, 4, 7.0, 1.0)
    lo, hi = slabs[1]
    d = SP.SlabDomain(model, g, lo, hi, halo, 1.0, 160, 80)
    assert d.origin == lo - halo
    assert d.box_local[0] > hi - lo + 2 * halo + h.rc_rad + 1.0 - 1e-3
    assert tuple(d.box_local[1:]) == (300.0, 300.0)
    assert d.local_cap >= N * (hi - lo + 2 * halo) / 300.0
    with pytest.raises(ValueError):
        SP.SlabDomain(model, SimpleNamespace(n_cfg=2, n_atoms=N, box_host=L, pos=g.pos), lo, hi, halo, 1.0, 160, 80)

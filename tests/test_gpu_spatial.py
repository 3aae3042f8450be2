"""Spatial decomposition (slabs along x with a two-layer halo) against the
whole-system evaluation, with the ranks emulated one after another on one
GPU: the owned atoms' forces, the energy and the virial; the selection
against a host recomputation; and three slabs against the FP64 oracle.

The owned atoms see the same neighbours as in the whole system, in another
list order.  FP32 sums in another order differ by a few ulp of the terms, so
forces agree to 1e-5 eV/A (terms are below ~1 eV/A).  The FP64 totals sum
FP32 per-atom values: 1e-6 eV per atom."""
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


def whole(nb, model, s, cap=112, cap_ang=56):
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang, shifts=False)
    ws = nb.Workspace(model, s.n_atoms, 1, cap, cap_ang)
    nb.neighbors(model, dsys, nl, SKIN, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    return dsys, nl, ws, nb.energy_forces_virial(model, dsys, nl, ws)


@pytest.mark.parametrize("world", [2, 3])
def test_slab_evaluation_matches_whole_system(nb, world):
    import torch
    from paper_2607_06969_gb300 import spatial as SP
    h = I.HYPER_SMALL
    s = I.rocksalt(14, vacancy=0.2, tag=6)
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys, _, _, (e_ref, f_ref, et_ref, v_ref) = whole(nb, model, s)
    slabs, halo = SP.plan_slabs(float(s.box[0, 0]), world, h.rc_rad, SKIN)
    doms = [SP.SlabDomain(model, dsys, lo, hi, halo, SKIN, 112, 56) for lo, hi in slabs]
    F = torch.zeros_like(f_ref)
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    V = torch.zeros(1, 9, dtype=torch.float64, device="cuda")
    owned = []
    for d in doms:
        d.rebuild()
        assert nb.check_list(d.nl) == nb.NEP_OK
        e, v = d.evaluate(F)
        E += e
        V += v
        owned.append(d.idx[:d.n_owned].cpu().numpy())
    owned = np.concatenate(owned)
    assert owned.size == s.n_atoms and np.array_equal(np.sort(owned), np.arange(s.n_atoms))
    assert (F - f_ref).abs().max().item() <= 1e-5
    assert abs(E.item() - et_ref.item()) <= 1e-6 * s.n_atoms
    assert (V - v_ref).abs().max().item() <= 1e-6 * s.n_atoms


def test_domain_select_against_host(nb):
    """Owned atoms and ghosts with their images, in atom order, against the
    same classification done on the host in FP32."""
    from paper_2607_06969_gb300 import spatial as SP
    h = I.HYPER_SMALL
    s = I.rocksalt(14, vacancy=0.2, tag=6)
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    Lx = np.float32(s.box[0, 0])
    slabs, halo = SP.plan_slabs(float(Lx), 3, h.rc_rad, SKIN)
    x = s.pos32()[:, 0].astype(np.float32)
    for lo, hi in slabs:
        d = SP.SlabDomain(model, dsys, lo, hi, halo, SKIN, 112, 56)
        n_owned, n_local = d._select()
        lo32, hi32, ha32 = np.float32(lo), np.float32(hi), np.float32(halo)
        own = np.nonzero((x >= lo32) & (x < hi32))[0]
        gh, im = [], []
        for i in np.setdiff1d(np.arange(x.size), own):
            for k in (-1, 0, 1):
                xs = np.float32(x[i] + np.float32(k) * Lx)
                if (lo32 - ha32 <= xs < lo32) or (hi32 <= xs < hi32 + ha32):
                    gh.append(i)
                    im.append(k)
                    break
        assert n_owned == own.size and n_local == own.size + len(gh)
        assert np.array_equal(d.idx[:n_local].cpu().numpy(), np.concatenate([own, gh]).astype(np.int32))
        assert np.array_equal(d.img[:n_local].cpu().numpy(), np.concatenate([np.zeros(own.size), im]).astype(np.int32))


def test_slab_evaluation_matches_oracle(nb):
    """Three slabs of a 12,442-atom rock-salt cell against the FP64 oracle:
    the owned atoms' E_i and F_i on a sample of atoms within 1 A of a slab
    face (their neighbourhoods reach furthest into the halo) and of atoms
    inside the slabs, at the FP32 parity bars (1e-6 eV, 1e-4 eV/A); the
    summed energy and virial against the oracle's whole-system values
    (1e-6 and 1e-5 eV per atom)."""
    import torch
    from paper_2607_06969_gb300 import spatial as SP
    h = I.HYPER_SMALL
    th32 = I.init_params(h).astype(np.float32)
    s = I.rocksalt(12, vacancy=0.2, tag=16)
    model = nb.Model(h, th32)
    gsys = nb.DeviceSystem.from_inputs(s)
    Lx = float(s.box[0, 0])
    slabs, halo = SP.plan_slabs(Lx, 3, h.rc_rad, SKIN)
    doms = [SP.SlabDomain(model, gsys, lo, hi, halo, SKIN, 112, 56) for lo, hi in slabs]
    F = torch.zeros(3, s.n_atoms, dtype=torch.float32, device="cuda")
    Ei = torch.zeros(s.n_atoms, dtype=torch.float32, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    V = torch.zeros(1, 9, dtype=torch.float64, device="cuda")
    for d in doms:
        d.rebuild()
        assert nb.check_list(d.nl) == nb.NEP_OK
        e, v = d.evaluate(F, e_atom_global=Ei)
        E += e
        V += v
    F = F.cpu().numpy().T.astype(np.float64)
    Ei = Ei.cpu().numpy().astype(np.float64)

    p32 = s.pos32()
    x = p32[:, 0].astype(np.float64)
    faces = np.array([lo for lo, _ in slabs] + [Lx])
    dface = np.abs(x[:, None] - faces[None, :]).min(1)
    rng = np.random.default_rng(16)
    edge = np.nonzero(dface < 1.0)[0]
    inner = np.nonzero(dface >= 1.0)[0]
    centers = np.concatenate([rng.choice(edge, 48, replace=False), rng.choice(inner, 16, replace=False)])
    box64 = s.box.astype(np.float32).astype(np.float64)
    ref = O.evaluate_centers(h, th32.astype(np.float64), p32, p32.astype(np.float64), s.types, box64,
                             s.atom_off, centers)
    c = ref["centers"]
    assert np.abs(Ei[c] - ref["E"]).max() <= 1e-6
    assert np.abs(F[c] - ref["F"]).max() <= 1e-4

    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    whole = O.energy_forces_virial(h, th32.astype(np.float64), p32.astype(np.float64), s.types, box64,
                                   s.atom_off, pairs)
    assert abs(E.item() - whole["Etot"][0]) <= 1e-6 * s.n_atoms
    assert np.abs(V.cpu().numpy().reshape(3, 3) - whole["V"][0]).max() <= 1e-5 * s.n_atoms
    assert np.abs(F - whole["F"]).max() <= 1e-4
    assert np.abs(Ei - whole["E"]).max() <= 1e-6

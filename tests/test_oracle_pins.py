"""Pins for the FP64 oracle: each test ties an oracle function to something
other than itself (a closed form, a library routine, a finite difference, an
invariant, a count the paper prints)."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb
from numpy.polynomial import legendre as npleg
from scipy import special

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

H0 = I.HYPER_SMALL


def tiny_hyper(**kw):
    base = dict(n_types=3, n_rad=3, n_ang=2, k_rad=4, k_ang=3, l_max=4, has_4body=1,
                n_hidden=4, rc_rad=5.0, rc_ang=4.0)
    base.update(kw)
    return I.Hyper(**base)


def iso_system(pos, types, L=60.0):
    """Atoms placed near the middle of a big periodic box (no image in range)."""
    pos = np.asarray(pos, np.float64) + L / 2
    return I.System(pos=pos, types=np.asarray(types, np.int32), box=np.array([[L, L, L]]),
                    atom_off=np.array([0, len(types)]))


def efv(h, theta, s, cutoff=None):
    pr = O.neighbor_pairs(s.pos.astype(np.float32), s.box, s.atom_off,
                          cutoff if cutoff is not None else h.rc_rad)
    return O.energy_forces_virial(h, theta, s.pos, s.types, s.box, s.atom_off, pr), pr


# --- counts the paper prints -----------------------------------------------
def test_param_count_table2_is_7p9k():
    # Section 4.1.2 / 4.2: the Table 2 NEP (n_R=10, n_A=8, N_basis 8/8,
    # l_max=4, 50 neurons, 3 species, 2+3-body) has 7.9k parameters.
    assert O.param_count(I.HYPER_TABLE2) == 7899
    assert O.descriptor_dim(I.HYPER_TABLE2) == 42


def test_descriptor_dim_small_is_38():
    # 216-atom workload: n_R=8, n_A=6, l_max=4 plus 4-body -> 38-dim
    assert O.descriptor_dim(H0) == 38
    assert O.param_count(H0) == H0.n_params == 4611


# --- radial functions --------------------------------------------------------
def test_cutoff_values():
    fc, dfc = O.cutoff_fn(np.array([0.0, 3.5, 7.0, 8.0]), 7.0)
    assert np.allclose(fc, [1.0, 0.5, 0.0, 0.0], atol=1e-15)
    assert abs(dfc[2]) < 1e-15


def test_chebyshev_basis_against_library_and_cosines():
    rc, K = 7.0, 8
    r = np.linspace(0.3, 6.99, 41)
    Q, dQ = O.chebyshev_basis(r, rc, K)
    x = 2 * (r / rc - 1) ** 2 - 1
    fc = 0.5 * (1 + np.cos(np.pi * r / rc))
    for k in range(K):
        Tk = npcheb.chebval(x, [0] * k + [1])
        assert np.allclose(Q[:, k], 0.5 * (Tk + 1) * fc, atol=1e-14)
        # T_k(cos phi) = cos(k phi)
        assert np.allclose(Tk, np.cos(k * np.arccos(x)), atol=1e-12)
    assert np.allclose(Q[:, 0], fc, atol=1e-15)           # f_0 = f_c
    h = 1e-6
    Qp, _ = O.chebyshev_basis(r + h, rc, K)
    Qm, _ = O.chebyshev_basis(r - h, rc, K)
    assert np.allclose(dQ, (Qp - Qm) / (2 * h), atol=1e-8)
    # every basis function and its slope vanish at the cutoff
    Qc, dQc = O.chebyshev_basis(np.array([rc - 1e-9]), rc, K)
    assert np.abs(Qc).max() < 1e-15 and np.abs(dQc).max() < 1e-7


def test_legendre_against_scipy():
    c = np.linspace(-1, 1, 17)
    P, dP = O.legendre(c, 4)
    for l in range(5):
        assert np.allclose(P[l], special.eval_legendre(l, c), atol=1e-14)
        der = npleg.legval(c, npleg.legder([0] * l + [1]))
        assert np.allclose(dP[l], der, atol=1e-13)


# --- descriptors: closed forms --------------------------------------------------
def g_closed(coef, r, rc):
    """g_n(r) = sum_k c[n][k] (T_k(x)+1)/2 f_c with T_k from numpy's chebval."""
    x = 2 * (r / rc - 1) ** 2 - 1
    fc = 0.5 * (1 + math.cos(math.pi * r / rc)) if r < rc else 0.0
    K = coef.shape[1]
    Q = np.array([0.5 * (npcheb.chebval(x, [0] * k + [1]) + 1) * fc for k in range(K)])
    return coef @ Q


def named_blocks(h, seed=11):
    """Random named parameter blocks, and theta assembled from them in the
    flat order that include/nep.h states: for t in types W0[t][H][D], b0[t][H],
    w1[t][H], b1[t]; then cR[Zi][Zj][n_rad][k_rad]; then cA[Zi][Zj][n_ang][k_ang]."""
    rng = np.random.default_rng(seed)
    T, H, D = h.n_types, h.n_hidden, O.descriptor_dim(h)
    blk = dict(W0=rng.normal(size=(T, H, D)), b0=rng.normal(size=(T, H)), w1=rng.normal(size=(T, H)),
               b1=rng.normal(size=T), cR=0.3 * rng.normal(size=(T, T, h.n_rad, h.k_rad)),
               cA=0.3 * rng.normal(size=(T, T, h.n_ang, h.k_ang)))
    parts = []
    for t in range(T):
        for r in range(H):                      # W0[t] row by row: hidden unit outer, descriptor inner
            parts += [blk["W0"][t, r, d] for d in range(D)]
        parts += list(blk["b0"][t]) + list(blk["w1"][t]) + [blk["b1"][t]]
    for a in range(T):
        for b in range(T):
            for n in range(h.n_rad):
                parts += list(blk["cR"][a, b, n])
    for a in range(T):
        for b in range(T):
            for n in range(h.n_ang):
                parts += list(blk["cA"][a, b, n])
    return blk, np.array(parts, np.float64)


def test_unpack_follows_the_header_block_order():
    """unpack maps the flat vector onto the named blocks in nep.h's order
    (H != D, so a transposed W0 cannot pass), and the energy computed from
    the named blocks by hand equals the oracle's: an isolated atom has q = 0
    and E = w1 . tanh(b0) + b1 (a swapped b0/w1 fails); a dimer's E uses W0
    and the ordered-pair radial and angular blocks."""
    h = tiny_hyper()
    blk, th = named_blocks(h)
    assert th.size == O.param_count(h)
    prm = O.unpack(h, th)
    for k in ("W0", "b0", "w1", "b1", "cR", "cA"):
        assert np.array_equal(getattr(prm, k), blk[k]), k
    for t in range(h.n_types):
        out, _ = efv(h, th, iso_system([[0, 0, 0]], [t]))
        assert abs(out["Etot"][0] - (blk["w1"][t] @ np.tanh(blk["b0"][t]) + blk["b1"][t])) < 1e-13
    r, ta, tb = 2.7, 0, 2
    out, _ = efv(h, th, iso_system([[0, 0, 0], [0, 0, r]], [ta, tb]))
    e = 0.0
    for a, b in ((ta, tb), (tb, ta)):
        gR = g_closed(blk["cR"][a, b], r, h.rc_rad)
        gA = g_closed(blk["cA"][a, b], r, h.rc_ang)
        qq = np.concatenate([gR, np.repeat(gA ** 2, h.l_max), 2.0 / 9.0 * gA ** 3])
        e += blk["w1"][a] @ np.tanh(blk["W0"][a] @ qq + blk["b0"][a]) + blk["b1"][a]
    assert abs(out["Etot"][0] - e) < 1e-12


@pytest.mark.parametrize("ta,tb", [(0, 2), (1, 1), (2, 0)])
def test_dimer_closed_form(ta, tb):
    h = H0
    th = I.init_params(h, seed=7)
    prm = O.unpack(h, th)
    r = 3.1
    s = iso_system([[0, 0, 0], [r * 0.6, r * 0.8, 0]], [ta, tb])
    out, _ = efv(h, th, s)
    q = out["q"]
    for a, b, row in ((ta, tb, 0), (tb, ta, 1)):
        gR = g_closed(prm.cR[a, b], r, h.rc_rad)
        gA = g_closed(prm.cA[a, b], r, h.rc_ang)
        assert np.allclose(q[row, :h.n_rad], gR, atol=1e-13)
        ang = q[row, h.n_rad:h.n_rad + h.n_ang * 4].reshape(h.n_ang, 4)
        assert np.allclose(ang, (gA ** 2)[:, None] * np.ones(4), atol=1e-13)   # P_l(1) = 1
        assert np.allclose(q[row, h.n_rad + h.n_ang * 4:], 2.0 / 9.0 * gA ** 3, atol=1e-14)
    # energy from the closed-form network, force = -dE/dr along the bond
    def etot(rr):
        e = 0.0
        for a, b in ((ta, tb), (tb, ta)):
            gR = g_closed(prm.cR[a, b], rr, h.rc_rad)
            gA = g_closed(prm.cA[a, b], rr, h.rc_ang)
            qq = np.concatenate([gR, np.repeat(gA ** 2, 4), 2.0 / 9.0 * gA ** 3])
            e += prm.w1[a] @ np.tanh(prm.W0[a] @ qq + prm.b0[a]) + prm.b1[a]
        return e
    assert abs(out["Etot"][0] - etot(r)) < 1e-12
    dEdr = (etot(r + 1e-6) - etot(r - 1e-6)) / 2e-6
    u = np.array([0.6, 0.8, 0.0])
    assert np.allclose(out["F"][1], -dEdr * u, atol=1e-8)
    assert np.allclose(out["F"][0], dEdr * u, atol=1e-8)


def test_trimer_angle_and_4body_triple_sum():
    h = H0
    th = I.init_params(h, seed=8)
    prm = O.unpack(h, th)
    r1, r2, ang = 2.9, 3.6, 1.1
    p1 = np.array([r1, 0, 0])
    p2 = r2 * np.array([math.cos(ang), math.sin(ang), 0])
    s = iso_system([[0, 0, 0], p1, p2], [2, 0, 1])
    out, _ = efv(h, th, s)
    q0 = out["q"][0]
    g1 = g_closed(prm.cA[2, 0], r1, h.rc_ang)
    g2 = g_closed(prm.cA[2, 1], r2, h.rc_ang)
    ang_q = q0[h.n_rad:h.n_rad + 4 * h.n_ang].reshape(h.n_ang, 4)
    for l in range(1, 5):
        want = g1 ** 2 + g2 ** 2 + 2 * g1 * g2 * special.eval_legendre(l, math.cos(ang))
        assert np.allclose(ang_q[:, l - 1], want, atol=1e-13)
    # q4_n = sum_jkm g g g [(a.b)(b.c)(c.a) - ((a.b)^2+(b.c)^2+(c.a)^2)/3 + 2/9]
    us = [p1 / r1, p2 / r2]
    gs = [g1, g2]
    want = np.zeros(h.n_ang)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                ab, bc, ca = us[a] @ us[b], us[b] @ us[c], us[c] @ us[a]
                want += gs[a] * gs[b] * gs[c] * (ab * bc * ca - (ab ** 2 + bc ** 2 + ca ** 2) / 3 + 2 / 9)
    assert np.allclose(q0[h.n_rad + 4 * h.n_ang:], want, atol=1e-14)


def test_legendre_form_equals_sform_addition_theorem():
    # q_nl = 4 pi/(2l+1) sum_m |sum_j g_n(r_j) Y_lm(rhat_j)|^2 (Eqs. 16-17)
    h = H0
    th = I.init_params(h, seed=9)
    prm = O.unpack(h, th)
    rng = np.random.default_rng(5)
    nb = 9
    dirs = rng.normal(size=(nb, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rs = rng.uniform(2.2, 4.9, size=nb)
    typ = rng.integers(0, 3, size=nb)
    s = iso_system(np.vstack([[0, 0, 0], dirs * rs[:, None]]), np.concatenate([[1], typ]))
    out, _ = efv(h, th, s)
    q0 = out["q"][0]
    G = np.array([g_closed(prm.cA[1, t], r, h.rc_ang) for t, r in zip(typ, rs)])   # [nb, n]
    theta = np.arccos(dirs[:, 2])
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    for l in range(1, 5):
        tot = np.zeros(h.n_ang)
        for m in range(-l, l + 1):
            Y = special.sph_harm_y(l, m, theta, phi)
            S = G.T @ Y
            tot += np.abs(S) ** 2
        tot *= 4 * np.pi / (2 * l + 1)
        assert np.allclose(q0[h.n_rad + (l - 1)::4][:h.n_ang], tot, atol=1e-12)


# --- forces and virial against finite differences ------------------------------
def small_periodic(seed=0, n=40, L=10.5):
    rng = I.rng_for(99, seed)
    p = I.rsa_pack(rng, n, L, 2.3)
    t = rng.integers(0, 3, size=n).astype(np.int32)
    return I.System(pos=p, types=t, box=np.array([[L, L * 1.05, L * 0.97]]),
                    atom_off=np.array([0, n]))


@pytest.mark.parametrize("hyp", ["tiny", "small"])
def test_forces_central_difference(hyp):
    h = tiny_hyper() if hyp == "tiny" else H0
    th = I.init_params(h, seed=11)
    s = small_periodic()            # box ~10.5 A < 2 rc: several images of one j
    pr = O.neighbor_pairs(s.pos.astype(np.float32), s.box, s.atom_off, h.rc_rad + 1.0)
    out = O.energy_forces_virial(h, th, s.pos, s.types, s.box, s.atom_off, pr)
    rng = np.random.default_rng(3)
    eps = 1e-5
    for _ in range(10):
        a, c = rng.integers(0, s.n_atoms), rng.integers(0, 3)
        pp = s.pos.copy(); pp[a, c] += eps
        pm = s.pos.copy(); pm[a, c] -= eps
        Ep = O.energy_forces_virial(h, th, pp, s.types, s.box, s.atom_off, pr)["Etot"][0]
        Em = O.energy_forces_virial(h, th, pm, s.types, s.box, s.atom_off, pr)["Etot"][0]
        fd = -(Ep - Em) / (2 * eps)
        assert abs(out["F"][a, c] - fd) < 1e-8 * max(1.0, abs(fd)), (a, c, out["F"][a, c], fd)
    assert np.abs(out["F"].sum(0)).max() < 1e-12


def test_virial_finite_strain():
    h = H0
    th = I.init_params(h, seed=12)
    s = small_periodic(seed=1)
    pr = O.neighbor_pairs(s.pos.astype(np.float32), s.box, s.atom_off, h.rc_rad + 1.0)
    out = O.energy_forces_virial(h, th, s.pos, s.types, s.box, s.atom_off, pr)
    i, j, sh = pr
    cfg = np.zeros(s.n_atoms, int)
    rij = O.pair_vectors(s.pos, s.box[cfg], i, j, sh)
    prm = O.unpack(h, th)

    def E_strained(eps_mat):
        r2 = rij @ (np.eye(3) + eps_mat).T
        _, E, _, _ = O.atom_terms(h, prm, s.types, np.arange(s.n_atoms), i, j, r2)
        return E.sum()

    d = 1e-6
    V_fd = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            e = np.zeros((3, 3)); e[a, b] = d
            V_fd[a, b] = -(E_strained(e) - E_strained(-e)) / (2 * d)
    assert np.allclose(out["V"][0], V_fd, atol=1e-7)
    assert np.allclose(out["V"][0], out["V"][0].T, atol=1e-12)


# --- invariances -----------------------------------------------------------------
def test_rotation_translation_permutation_invariance():
    h = H0
    th = I.init_params(h, seed=13)
    rng = np.random.default_rng(1)
    cl = I.rsa_pack(rng, 30, 9.0, 2.4) - 4.5
    t = rng.integers(0, 3, size=30).astype(np.int32)
    base, _ = efv(h, th, iso_system(cl, t))
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    rot, _ = efv(h, th, iso_system(cl @ Q.T, t))
    assert abs(rot["Etot"][0] - base["Etot"][0]) < 1e-12
    assert np.allclose(rot["F"], base["F"] @ Q.T, atol=1e-12)
    # translation inside a periodic box (atoms re-wrapped)
    s = small_periodic(seed=2)
    e0, _ = efv(h, th, s)
    s2 = I.System(pos=np.mod(s.pos + np.array([3.3, -1.7, 5.2]), s.box[0]), types=s.types,
                  box=s.box, atom_off=s.atom_off)
    e1, _ = efv(h, th, s2)
    assert abs(e0["Etot"][0] - e1["Etot"][0]) < 1e-11
    assert np.allclose(e0["E"], e1["E"], atol=1e-12)
    # permuting atoms (species travel with them) permutes E_i and F_i
    perm = np.random.default_rng(4).permutation(s.n_atoms)
    s3 = I.System(pos=s.pos[perm], types=s.types[perm], box=s.box, atom_off=s.atom_off)
    e3, _ = efv(h, th, s3)
    assert np.allclose(e3["E"], e0["E"][perm], atol=1e-12)
    assert np.allclose(e3["F"], e0["F"][perm], atol=1e-12)


# --- neighbours -------------------------------------------------------------------
def test_neighbors_against_kdtree_and_bins():
    from scipy.spatial import cKDTree
    s = I.rocksalt(10, vacancy=0.2, tag=77)     # 7,200 atoms, box 60 A: binned path
    p32 = s.pos32()
    L = float(s.box[0, 0])
    centers = np.arange(0, s.n_atoms, 97)
    i, j, sh = O.neighbor_pairs(p32, s.box, s.atom_off, 8.0, centers=centers)
    tree = cKDTree(p32.astype(np.float64), boxsize=L)
    for c in centers[:25]:
        nb = tree.query_ball_point(p32[c].astype(np.float64), 8.0 + 1e-4)
        d = np.array([np.linalg.norm((p32[k] - p32[c] + L / 2) % L - L / 2) for k in nb])
        sure = set(k for k, dd in zip(nb, d) if dd < 8.0 - 1e-4 and k != c)
        got = set(j[i == c].tolist())
        assert sure <= got and got <= set(nb) - {c}
    # brute force over all atoms of a sub-box gives the same lists as the binned path
    sub = centers[:8]
    ib, jb, sb = O.neighbor_pairs(p32, s.box, s.atom_off, 8.0, centers=sub)
    for c in sub:
        d = p32 - p32[c]
        shift = -np.round(d / L)
        dd = (d + (shift * L).astype(np.float32)).astype(np.float32)
        d2 = (dd[:, 0] * dd[:, 0] + dd[:, 1] * dd[:, 1]) + dd[:, 2] * dd[:, 2]
        want = set(np.nonzero(d2 < np.float32(64.0))[0].tolist()) - {int(c)}
        assert set(jb[ib == c].tolist()) == want


def test_neighbors_small_box_counts_images():
    # L = 9.04 A with a cutoff beyond L: one j is a neighbour through several
    # images, and an atom neighbours its own images.
    rng = np.random.default_rng(2)
    L = 9.04
    n = 24
    p = I.rsa_pack(rng, n, L, 2.4)
    s = I.System(pos=p, types=np.zeros(n, np.int32), box=np.array([[L, L, L]]),
                 atom_off=np.array([0, n]))
    p32 = s.pos32()
    rc = 9.5                                   # > L: self images and |s| = 2 images
    i, j, sh = O.neighbor_pairs(p32, s.box, s.atom_off, rc)
    # independent FP64 enumeration of images, with a band that excludes ties
    cnt_sure, cnt_max = np.zeros(n, int), np.zeros(n, int)
    for a in range(n):
        for b in range(n):
            for sx in range(-3, 4):
                for sy in range(-3, 4):
                    for sz in range(-3, 4):
                        if a == b and sx == sy == sz == 0:
                            continue
                        d = np.linalg.norm(p32[b].astype(float) - p32[a] + np.array([sx, sy, sz]) * L)
                        cnt_sure[a] += d < rc - 1e-4
                        cnt_max[a] += d < rc + 1e-4
    got = np.bincount(i, minlength=n)
    assert np.all(got >= cnt_sure) and np.all(got <= cnt_max)
    assert np.any((i == j))                     # self images present
    # the list is symmetric: (i, j, s) present <=> (j, i, -s) present
    fwd = set(zip(i.tolist(), j.tolist(), map(tuple, sh.tolist())))
    for a, b, t in fwd:
        assert (b, a, tuple(-np.array(t))) in fwd


# --- loss and gradient ----------------------------------------------------------------
def batch_case(h, n_cfg=3, seed=0):
    s = I.packing_batch([24, 31, 40][:n_cfg], tag=50 + seed)
    pr = O.neighbor_pairs(s.pos32(), s.box, s.atom_off, h.rc_rad)
    return s, pr


def test_loss_closed_form():
    h = tiny_hyper()
    th = I.init_params(h, seed=21)
    s, pr = batch_case(h)
    pos = s.pos32().astype(np.float64)
    out = O.energy_forces_virial(h, th, pos, s.types, s.box, s.atom_off, pr)
    B = s.n_cfg
    Nb = np.diff(s.atom_off).astype(float)
    dE, dF, dV = np.array([0.3, -0.2, 0.5]), 0.05, np.arange(9.0).reshape(3, 3) * 0.01
    L0 = O.loss_value(h, th, pos, s.types, s.box, s.atom_off, pr, out["Etot"] - dE,
                      out["F"] - dF, out["V"] - dV, mode=0)
    want = np.mean(1.0 * (dE / Nb) ** 2 + 1.0 * dF ** 2 + 0.1 * (dV ** 2).sum() / 9 / Nb ** 2)
    assert abs(L0 - want) < 1e-14
    L1 = O.loss_value(h, th, pos, s.types, s.box, s.atom_off, pr, out["Etot"] - dE,
                      out["F"] - dF, out["V"] - dV, mode=1)
    want1 = np.mean(dE ** 2 / Nb + dF ** 2 + 0.1 * (dV ** 2).sum() / 9 / Nb)
    assert abs(L1 - want1) < 1e-13
    zero = O.loss_value(h, th, pos, s.types, s.box, s.atom_off, pr, out["Etot"], out["F"], out["V"])
    assert abs(zero) < 1e-28


def test_loss_with_an_empty_configuration():
    """An empty configuration adds no loss term, whatever its labels, but
    counts in the batch size: inserting one into a batch of B scales the
    loss and its gradient by B / (B + 1), in both modes."""
    h = tiny_hyper()
    th = I.init_params(h, seed=29)
    s, pr = batch_case(h)
    pos = s.pos32().astype(np.float64)
    lab = O.energy_forces_virial(h, I.init_params(h, seed=30), pos, s.types, s.box, s.atom_off, pr)
    off2 = np.insert(s.atom_off, 1, s.atom_off[1])                     # empty configuration 1
    box2 = np.insert(s.box, 1, [20.0, 20.0, 20.0], axis=0)
    pr2 = O.neighbor_pairs(s.pos32(), box2, off2, h.rc_rad)
    E2 = np.insert(lab["Etot"], 1, 3.0)
    V2 = np.insert(lab["V"].reshape(-1, 9), 1, np.arange(9.0), axis=0)
    B = s.n_cfg
    for mode in (0, 1):
        def L1(t):
            return O.loss_value(h, t, pos, s.types, s.box, s.atom_off, pr, lab["Etot"], lab["F"], lab["V"],
                                mode=mode)

        def L2(t):
            return O.loss_value(h, t, pos, s.types, box2, off2, pr2, E2, lab["F"], V2, mode=mode)
        assert abs(L2(th) - L1(th) * B / (B + 1)) <= 1e-14 * abs(L1(th))
        idx = [0, 7, O.param_count(h) - 1]
        assert np.allclose(O.complex_step_grad(L2, th, idx), O.complex_step_grad(L1, th, idx) * B / (B + 1),
                           rtol=1e-12, atol=0)


def test_gradient_complex_step_vs_central_difference():
    h = tiny_hyper()
    th = I.init_params(h, seed=22)
    s, pr = batch_case(h)
    pos = s.pos32().astype(np.float64)
    teacher = I.init_params(h, seed=23)
    lab = O.energy_forces_virial(h, teacher, pos, s.types, s.box, s.atom_off, pr)

    def Lf(t):
        return O.loss_value(h, t, pos, s.types, s.box, s.atom_off, pr, lab["Etot"], lab["F"], lab["V"])

    P = O.param_count(h)
    idx = list(range(0, P, max(1, P // 25))) + [P - 1]
    g = O.complex_step_grad(Lf, th, idx)
    hh = 1e-4
    for a, k in enumerate(idx):
        tp, tm = th.copy(), th.copy()
        tp[k] += hh; tm[k] -= hh
        fd = (Lf(tp) - Lf(tm)) / (2 * hh)
        assert abs(g[a] - fd) <= 1e-6 * max(abs(fd), 1e-3), (k, g[a], fd)


def test_gradient_without_4body_mode1_complex_step_vs_central_difference():
    """The paper's own 2+3-body form (no 4-body term) under the printed loss
    (mode 1, Eqs. 19-21): the complex-step gradient against central FD."""
    h = tiny_hyper(has_4body=0)
    th = I.init_params(h, seed=26)
    s, pr = batch_case(h, seed=1)
    pos = s.pos32().astype(np.float64)
    lab = O.energy_forces_virial(h, I.init_params(h, seed=27), pos, s.types, s.box, s.atom_off, pr)

    def Lf(t):
        return O.loss_value(h, t, pos, s.types, s.box, s.atom_off, pr, lab["Etot"], lab["F"], lab["V"],
                            w=(0.5, 2.0, 0.3), mode=1)

    P = O.param_count(h)
    assert P == 3 * (h.n_hidden * (h.n_rad + 4 * h.n_ang) + 2 * h.n_hidden + 1) + 9 * (
        h.n_rad * h.k_rad + h.n_ang * h.k_ang)
    idx = list(range(0, P, max(1, P // 20))) + [P - 1]
    g = O.complex_step_grad(Lf, th, idx)
    for a, k in enumerate(idx):
        tp, tm = th.copy(), th.copy()
        tp[k] += 1e-4
        tm[k] -= 1e-4
        fd = (Lf(tp) - Lf(tm)) / 2e-4
        assert abs(g[a] - fd) <= 1e-6 * max(abs(fd), 1e-3), (k, g[a], fd)


def test_force_and_virial_adjoints_are_one_energy_tangent():
    """lam.F + mu:V (Eqs. 3-4) equals the derivative of the energy along the
    pair-vector tangent dr_ij = -(lam_j - lam_i) - mu r_ij: the identity the
    training backward evaluates instead of differentiating F and V."""
    h = tiny_hyper()
    th = I.init_params(h, seed=28)
    s = small_periodic(seed=3)
    pr = O.neighbor_pairs(s.pos.astype(np.float32), s.box, s.atom_off, h.rc_rad + 1.0)
    out = O.energy_forces_virial(h, th, s.pos, s.types, s.box, s.atom_off, pr)
    rng = np.random.default_rng(9)
    lam = rng.normal(size=(s.n_atoms, 3))
    mu = rng.normal(size=(3, 3))
    i, j, sh = pr
    rij = O.pair_vectors(s.pos, s.box[np.zeros(s.n_atoms, int)], i, j, sh)
    drij = -(lam[j] - lam[i]) - rij @ mu.T
    prm = O.unpack(h, th)

    def E(eps):
        return O.atom_terms(h, prm, s.types, np.arange(s.n_atoms), i, j, rij + eps * drij)[1].sum()

    d = 1e-6
    fd = (E(d) - E(-d)) / (2 * d)
    want = (lam * out["F"]).sum() + (mu * out["V"][0]).sum()
    assert abs(fd - want) < 1e-7 * max(1.0, abs(want)), (fd, want)


def test_adjoint_functional_gives_loss_gradient():
    # dL/dtheta = dPhi/dtheta with aE = dL/dE, lam = dL/dF, mu = dL/dV held fixed
    h = tiny_hyper()
    th = I.init_params(h, seed=24)
    s, pr = batch_case(h)
    pos = s.pos32().astype(np.float64)
    lab = O.energy_forces_virial(h, I.init_params(h, seed=25), pos, s.types, s.box, s.atom_off, pr)
    out = O.energy_forces_virial(h, th, pos, s.types, s.box, s.atom_off, pr)
    B = s.n_cfg
    Nb = np.diff(s.atom_off).astype(float)
    cfg = s.cfg_of_atom()
    aE = 2 * (out["Etot"] - lab["Etot"]) / Nb ** 2 / B
    lam = 2 * (out["F"] - lab["F"]) / (3 * Nb[cfg])[:, None] / B
    mu = 0.1 * 2 * (out["V"] - lab["V"]) / 9 / (Nb ** 2)[:, None, None] / B
    P = O.param_count(h)
    idx = list(range(0, P, 7))
    gL = O.complex_step_grad(lambda t: O.loss_value(h, t, pos, s.types, s.box, s.atom_off, pr,
                                                     lab["Etot"], lab["F"], lab["V"]), th, idx)
    gP = O.complex_step_grad(lambda t: O.adjoint_functional(h, t, pos, s.types, s.box, s.atom_off,
                                                            pr, aE, lam, mu), th, idx)
    assert np.allclose(gL, gP, rtol=1e-10, atol=1e-16)


# --- input generators ------------------------------------------------------------
def test_generators_composition():
    s, h = I.workload_cell216()
    assert s.n_atoms == 216 and np.bincount(s.types).tolist() == [54, 54, 108]
    s = I.rocksalt(5, vacancy=0.2, tag=9)
    assert np.bincount(s.types).tolist() == [200, 200, 500]
    b = I.packing_batch([24, 100], tag=9)
    from scipy.spatial import cKDTree
    for k in range(2):
        P = b.pos[b.atom_off[k]:b.atom_off[k + 1]]
        d, _ = cKDTree(P, boxsize=b.box[k, 0]).query(P, k=2)
        assert d[:, 1].min() >= 2.4
    assert np.isclose(b.box[1, 0], (100 / 0.0325) ** (1 / 3))


def test_workload_sizes():
    """The synthetic workloads have the sizes the workload definitions state:
    216 atoms; 900,000 atoms in a 300 A box; 3,686,400 atoms in a 480 A box;
    128 configurations of 24-512 atoms (mean about 268); 1,024 replicas of
    64-4096 atoms, log-uniform (about 1.0M atoms)."""
    s, h = I.workload_cell216()
    assert s.n_atoms == 216 and np.allclose(s.box, 18.0) and O.descriptor_dim(h) == 38
    s, _ = I.workload_md900k()
    assert s.n_atoms == 900_000 and np.allclose(s.box, 300.0)
    assert np.bincount(s.types).tolist() == [200_000, 200_000, 500_000]     # 20% of 500,000 cation sites vacant
    del s
    s, h = I.workload_mixed3m7()
    assert s.n_atoms == 3_686_400 and np.allclose(s.box, 480.0) and h.n_hidden == 64
    del s
    c = np.asarray(I.uniform_counts(128, 24, 512, tag=2))
    assert c.min() >= 24 and c.max() <= 512 and abs(c.mean() - 268) < 25
    c = np.asarray(I.loguniform_counts(1024, 64, 4096, tag=4))
    assert c.min() >= 64 and c.max() <= 4096 and abs(c.sum() - 1.0e6) < 0.1e6
    assert abs(np.median(np.log(c)) - 0.5 * (np.log(64) + np.log(4096))) < 0.2     # log-uniform


def test_velocities_temperature_momentum_and_units():
    """The MD start: Maxwell-Boltzmann velocities at T with zero momentum per
    configuration, and the unit constants against CODATA 2018 (1 u A^2/fs^2
    in eV, and k_B in eV/K)."""
    assert abs(I.MVV_TO_EV - 1.66053906660e-27 * 1e-20 / 1e-30 / 1.602176634e-19) < 1e-4
    assert abs(I.KB_EV - 1.380649e-23 / 1.602176634e-19) < 1e-12
    types = np.repeat(np.array([0, 1, 2], np.int32), 20000)
    np.random.default_rng(2).shuffle(types)
    off = np.array([0, 25000, 25000, 60000])                       # one empty configuration
    v = I.maxwell_boltzmann(types, 900.0, atom_off=off)
    m = I.MASSES[types]
    for b in (0, 2):
        s = slice(off[b], off[b + 1])
        p = (m[s, None] * v[s]).sum(0)
        assert np.abs(p).max() < 1e-9 * np.sqrt((m[s, None] * v[s] ** 2).sum())
        n = off[b + 1] - off[b]
        T = (m[s, None] * v[s] ** 2).sum() * I.MVV_TO_EV / (3 * (n - 1) * I.KB_EV)
        assert abs(T - 900.0) < 0.02 * 900.0, T


def test_evaluate_centers_equals_whole_system():
    """The neighbourhood evaluation of sampled atoms (used at the full
    workload sizes) against the whole-system evaluation (pinned above by
    finite differences and invariances): the same E_i and F_i, and per-atom
    virials that sum to each configuration's virial."""
    s = I.packing_batch([24, 40], tag=77)
    h = tiny_hyper()
    th = I.init_params(h)
    p32 = s.pos32()
    box64 = s.box.astype(np.float32).astype(np.float64)
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    whole = O.energy_forces_virial(h, th, p32.astype(np.float64), s.types, box64, s.atom_off, pairs)
    centers = np.arange(s.n_atoms)
    part = O.evaluate_centers(h, th, p32, p32.astype(np.float64), s.types, box64, s.atom_off, centers)
    assert np.allclose(part["E"], whole["E"], rtol=0, atol=1e-12)
    assert np.allclose(part["F"], whole["F"], rtol=0, atol=1e-12)
    for b in range(s.n_cfg):
        a0, a1 = s.atom_off[b], s.atom_off[b + 1]
        assert np.allclose(part["W"][a0:a1].sum(0), whole["V"][b], rtol=0, atol=1e-11)
    # a sample of centres gives the same rows as the full evaluation
    sub = O.evaluate_centers(h, th, p32, p32.astype(np.float64), s.types, box64, s.atom_off,
                             np.array([3, 30, 50]))
    assert np.allclose(sub["F"], whole["F"][[3, 30, 50]], rtol=0, atol=1e-12)

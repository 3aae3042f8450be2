"""FP64 CPU oracle for the NEP per-atom path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline/reference leg
may import this module.  It shares no code, header, table or constant with the
CUDA path in paper_2607_06969_gb300/, and it imports nothing from it.

What it computes, in the paper's order and notation (AI2Pot, Section 2):

* Eq. 1   E_tot = sum_i E_i
* Eq. 2   E_i = f_theta({q}), a single-hidden-layer tanh network per species
          (Section 2.3): E_i = sum_h w1[h] tanh(sum_d W0[h][d] q_d + b0[h]) + b1
* Eq. 3   F_i = sum_j (dE_i/dr_ij - dE_j/dr_ji), r_ij = r_j - r_i
* Eq. 4   V_ab = - sum_i sum_j dE_i/dr_ij,a r_ij,b
* Eq. 11  q_n = sum_j sum_k cR[Zi][Zj][n][k] Q_k(r_ij)
* Eqs. 12-15  Q_k(r) = (T_k(x)+1)/2 f_c(r),  x = 2(r/rc-1)^2-1,
              f_c = (1+cos(pi r/rc))/2 for r < rc, else 0 (both give 0 at rc)
* Eqs. 16-17  q_nl = sum_m C_lm S_nlm^2; written here in its Legendre form
          q_nl = sum_j sum_k g_n(r_ij) g_n(r_ik) P_l(rhat_ij . rhat_ik),
          which equals Eq. 17 by the addition theorem of spherical harmonics
          (C_lm = 4 pi/(2l+1) for orthonormal real harmonics), l = 1..l_max.
* 4-body  the paper's NEP stops at 3-body terms (Section 2.3); the 4-body
          descriptor used here is q4_n = tr(A_n^3) with
          A_n = sum_j g_n(r_ij) (rhat rhat^T - I/3), the cubic invariant of
          the l = 2 coupling.
* Eqs. 18-21  loss (mode 1), and the per-atom-normalised batch loss (mode 0):
          L = 1/B sum_b [wE (dE_b/N_b)^2 + wF/(3 N_b) sum |dF|^2
                         + wV/9 sum (dV_b/N_b)^2].
* Section 3.3.1  the optimiser: Adam with beta1 = 0.9, beta2 = 0.999,
          eps = 1e-8 and no weight decay (Kingma and Ba's update with bias
          corrections).

Readings where the paper is silent: n runs 0..n_max-1 and l runs 1..l_max
(no l = 0); k runs 0..N_basis-1; c is indexed by the ordered species pair;
no descriptor scaling; cutoff is strict (r < rc).  The parameter gradient is
taken by complex-step differentiation (Squire & Trapp 1998) through the
analytic force code: every step below is complex-analytic in the parameters.

Pins for every function live in tests/test_oracle_pins.py, tests/test_train_loop.py
and tests/test_golden.py; tests/test_oracle_mutations.py shows that they bind.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

L_MAX = 4


# ---------------------------------------------------------------------------
# parameter layout
# ---------------------------------------------------------------------------
def descriptor_dim(h) -> int:
    """D = n_rad + n_ang * l_max + n_ang * has_4body (Section 2.3)."""
    return h.n_rad + h.n_ang * h.l_max + (h.n_ang if h.has_4body else 0)


def param_count(h) -> int:
    D, H, T = descriptor_dim(h), h.n_hidden, h.n_types
    return T * (H * D + H + H + 1) + T * T * (h.n_rad * h.k_rad + h.n_ang * h.k_ang)


@dataclass
class Params:
    W0: np.ndarray   # [T, H, D]
    b0: np.ndarray   # [T, H]
    w1: np.ndarray   # [T, H]
    b1: np.ndarray   # [T]
    cR: np.ndarray   # [T, T, n_rad, k_rad]
    cA: np.ndarray   # [T, T, n_ang, k_ang]


def unpack(h, theta: np.ndarray) -> Params:
    D, H, T = descriptor_dim(h), h.n_hidden, h.n_types
    assert theta.size == param_count(h), (theta.size, param_count(h))
    o = 0
    W0, b0, w1, b1 = [], [], [], []
    for _ in range(T):
        W0.append(theta[o:o + H * D].reshape(H, D)); o += H * D
        b0.append(theta[o:o + H]); o += H
        w1.append(theta[o:o + H]); o += H
        b1.append(theta[o:o + 1]); o += 1
    nR = T * T * h.n_rad * h.k_rad
    cR = theta[o:o + nR].reshape(T, T, h.n_rad, h.k_rad); o += nR
    nA = T * T * h.n_ang * h.k_ang
    cA = theta[o:o + nA].reshape(T, T, h.n_ang, h.k_ang); o += nA
    return Params(np.stack(W0), np.stack(b0), np.stack(w1), np.concatenate(b1), cR, cA)


# ---------------------------------------------------------------------------
# neighbours: all (j, image s) != (i, 0) with |r_j + s*L - r_i| < rc,
# decided by a fixed FP32 predicate:
#   dx = (x_j - x_i) + s_x L_x ;  d2 = (dx dx + dy dy) + dz dz ;  d2 < fl32(rc rc)
# ---------------------------------------------------------------------------
def _pred_f32(pi, pj, s, L32, rc2):
    """pi [M,3], pj [M,3] float32, s [M,3] int, L32 [3] float32 -> mask."""
    d = (pj - pi) + s.astype(np.float32) * L32
    d = d.astype(np.float32)
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    return d2 < rc2


def neighbor_pairs(pos32: np.ndarray, box: np.ndarray, atom_off: np.ndarray, cutoff: float,
                   centers: np.ndarray | None = None):
    """Return (i, j, s[3]) int arrays, sorted by (i, j, sx, sy, sz).

    pos32 must be float32 positions wrapped into [0, L).  cutoff is rounded
    to float32 and squared in float32.  centers restricts the i's (global
    indices).  Every image |s_a| <= ceil(cutoff/L_a) is tested."""
    pos32 = np.asarray(pos32, np.float32)
    rc32 = np.float32(cutoff)
    rc2 = np.float32(rc32 * rc32)
    out_i, out_j, out_s = [], [], []
    B = box.shape[0]
    cent_mask = None
    if centers is not None:
        cent_mask = np.zeros(pos32.shape[0], bool)
        cent_mask[np.asarray(centers)] = True
    for b in range(B):
        a0, a1 = int(atom_off[b]), int(atom_off[b + 1])
        if a1 == a0:
            continue
        L32 = np.asarray(box[b], np.float32)
        P = pos32[a0:a1]
        n = a1 - a0
        ci = np.arange(n) if cent_mask is None else np.nonzero(cent_mask[a0:a1])[0]
        if ci.size == 0:
            continue
        S = [int(math.ceil(float(rc32) / float(L32[a]))) for a in range(3)]
        imgs = np.array([(x, y, z) for x in range(-S[0], S[0] + 1)
                         for y in range(-S[1], S[1] + 1)
                         for z in range(-S[2], S[2] + 1)], np.int64)
        ncell = [int(np.floor(float(L32[a]) / (float(rc32) + 0.01))) for a in range(3)]
        use_bins = min(ncell) >= 3 and n > 4096
        # every edge longer than 2 rc: at most one image of j lies within rc,
        # the minimum image, so that single image is tested
        single = (not use_bins) and all(float(L32[a]) > 2.0 * float(rc32) + 0.01 for a in range(3))
        if single:
            for c0 in range(0, ci.size, 64):
                ii = ci[c0:c0 + 64]
                I = np.repeat(ii, n)
                J = np.tile(np.arange(n), ii.size)
                d = P[J].astype(np.float64) - P[I].astype(np.float64)
                Sx = -np.rint(d / L32.astype(np.float64)).astype(np.int64)
                keep = ~((I == J) & (Sx == 0).all(1))
                I, J, Sx = I[keep], J[keep], Sx[keep]
                m = _pred_f32(P[I], P[J], Sx, L32, rc2)
                out_i.append(I[m] + a0)
                out_j.append(J[m] + a0)
                out_s.append(Sx[m])
            continue
        if use_bins:
            cs = np.array([float(L32[a]) / ncell[a] for a in range(3)])
            cidx = np.minimum((P.astype(np.float64) / cs).astype(np.int64), np.array(ncell) - 1)
            flat = (cidx[:, 0] * ncell[1] + cidx[:, 1]) * ncell[2] + cidx[:, 2]
            order = np.argsort(flat, kind="stable")
            starts = np.searchsorted(flat[order], np.arange(ncell[0] * ncell[1] * ncell[2] + 1))
        for c0 in range(0, ci.size, 256 if not use_bins else 1):
            ii = ci[c0:c0 + (256 if not use_bins else 1)]
            if use_bins:
                i0 = ii[0]
                cands = []
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dz in (-1, 0, 1):
                            c = ((cidx[i0, 0] + dx) % ncell[0], (cidx[i0, 1] + dy) % ncell[1],
                                 (cidx[i0, 2] + dz) % ncell[2])
                            f = (c[0] * ncell[1] + c[1]) * ncell[2] + c[2]
                            cands.append(order[starts[f]:starts[f + 1]])
                jj_all = np.unique(np.concatenate(cands))
                I = np.repeat(ii, jj_all.size * imgs.shape[0])
                J = np.tile(np.repeat(jj_all, imgs.shape[0]), ii.size)
                Sx = np.tile(imgs, (ii.size * jj_all.size, 1))
            else:
                jj_all = np.arange(n)
                I = np.repeat(ii, n * imgs.shape[0])
                J = np.tile(np.repeat(jj_all, imgs.shape[0]), ii.size)
                Sx = np.tile(imgs, (ii.size * n, 1))
            keep = ~((I == J) & (Sx == 0).all(1))
            I, J, Sx = I[keep], J[keep], Sx[keep]
            m = _pred_f32(P[I], P[J], Sx, L32, rc2)
            out_i.append(I[m] + a0)
            out_j.append(J[m] + a0)
            out_s.append(Sx[m])
    if not out_i:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3), np.int64)
    i = np.concatenate(out_i)
    j = np.concatenate(out_j)
    s = np.concatenate(out_s)
    order = np.lexsort((s[:, 2], s[:, 1], s[:, 0], j, i))
    return i[order], j[order], s[order]


# ---------------------------------------------------------------------------
# radial functions (Eqs. 12-15)
# ---------------------------------------------------------------------------
def cutoff_fn(r, rc):
    """f_c = (1 + cos(pi r/rc))/2 inside, 0 outside (Eq. 14-15), and d f_c/dr."""
    inside = r < rc
    fc = np.where(inside, 0.5 * (1.0 + np.cos(np.pi * r / rc)), 0.0)
    dfc = np.where(inside, -0.5 * np.pi / rc * np.sin(np.pi * r / rc), 0.0)
    return fc, dfc


def chebyshev_basis(r, rc, K):
    """Q_k(r) = (T_k(x)+1)/2 f_c(r), x = 2(r/rc-1)^2-1 (Eqs. 12-13), k = 0..K-1,
    and dQ_k/dr.  T_k by the three-term recurrence T_{k+1} = 2x T_k - T_{k-1},
    T_k' by T'_{k+1} = 2 T_k + 2x T'_k - T'_{k-1}."""
    r = np.asarray(r, np.float64)
    fc, dfc = cutoff_fn(r, rc)
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    dx = 4.0 * (r / rc - 1.0) / rc
    T = np.zeros(r.shape + (K,))
    dT = np.zeros(r.shape + (K,))
    T[..., 0] = 1.0
    if K > 1:
        T[..., 1] = x
        dT[..., 1] = 1.0
    for k in range(1, K - 1):
        T[..., k + 1] = 2.0 * x * T[..., k] - T[..., k - 1]
        dT[..., k + 1] = 2.0 * T[..., k] + 2.0 * x * dT[..., k] - dT[..., k - 1]
    Q = 0.5 * (T + 1.0) * fc[..., None]
    dQ = 0.5 * dT * dx[..., None] * fc[..., None] + 0.5 * (T + 1.0) * dfc[..., None]
    return Q, dQ


def legendre(c, L):
    """P_l(c) and P_l'(c) for l = 0..L by Bonnet's recursion
    l P_l = (2l-1) c P_{l-1} - (l-1) P_{l-2} and P'_l = P'_{l-2} + (2l-1) P_{l-1}."""
    P = [np.ones_like(c), c]
    dP = [np.zeros_like(c), np.ones_like(c)]
    for l in range(2, L + 1):
        P.append(((2 * l - 1) * c * P[l - 1] - (l - 1) * P[l - 2]) / l)
        dP.append(dP[l - 2] + (2 * l - 1) * P[l - 1])
    return P, dP


# ---------------------------------------------------------------------------
# per-atom terms
# ---------------------------------------------------------------------------
def _segsum(vals, idx, n):
    """sum of vals rows grouped by idx (sorted) into n bins."""
    out = np.zeros((n,) + vals.shape[1:], dtype=vals.dtype)
    if vals.shape[0] == 0:
        return out
    starts = np.nonzero(np.r_[True, idx[1:] != idx[:-1]])[0]
    out[idx[starts]] = np.add.reduceat(vals, starts, axis=0)
    return out


def _type_pair_apply(coef, ti, tj, X):
    """out[p] = coef[ti[p], tj[p]] @ X[p]  (coef [T,T,n,K], X [P,K]) -> [P,n]."""
    T = coef.shape[0]
    out = np.zeros((X.shape[0], coef.shape[2]), dtype=np.result_type(coef, X))
    for a in range(T):
        for b in range(T):
            sel = (ti == a) & (tj == b)
            if sel.any():
                out[sel] = X[sel] @ coef[a, b].T
    return out


def pair_vectors(pos, box_of_atom, i, j, s):
    """r_ij = r_j + s*L - r_i in FP64 (Eq. 3's r_ij = r_j - r_i with images)."""
    return (pos[j] - pos[i]) + s * box_of_atom[i]


def atom_terms(h, prm: Params, types, owners, i, j, rij, chunk=2048):
    """For the owner atoms (sorted unique global ids) and their pairs (i in
    owners, sorted by i): descriptors q [n_own, D], energies E [n_own],
    dE/dq p [n_own, D] and pair derivatives f_ij = dE_i/dr_ij [P, 3]."""
    n_own = owners.size
    loc = np.searchsorted(owners, i)
    assert np.all(owners[loc] == i)
    ti, tj = types[i], types[j]
    r = np.sqrt((rij * rij).sum(1))
    u = rij / r[:, None]
    cdt = np.result_type(prm.cR, prm.W0, np.float64)
    D = descriptor_dim(h)
    L = h.l_max
    nA = h.n_ang

    # radial (Eq. 11)
    inR = r < h.rc_rad
    QR, dQR = chebyshev_basis(np.where(inR, r, h.rc_rad), h.rc_rad, h.k_rad)
    gR = _type_pair_apply(prm.cR, ti, tj, QR)
    dgR = _type_pair_apply(prm.cR, ti, tj, dQR)
    q = np.zeros((n_own, D), dtype=cdt)
    q[:, :h.n_rad] = _segsum(gR, loc, n_own)

    # angular pairs (r < rc_ang), grouped per owner and padded
    inA = r < h.rc_ang
    pa = np.nonzero(inA)[0]
    QA, dQA = chebyshev_basis(r[pa], h.rc_ang, h.k_ang)
    gA = _type_pair_apply(prm.cA, ti[pa], tj[pa], QA)
    dgA = _type_pair_apply(prm.cA, ti[pa], tj[pa], dQA)
    locA = loc[pa]
    cntA = np.bincount(locA, minlength=n_own)
    firstA = np.concatenate([[0], np.cumsum(cntA)])
    slotA = np.arange(pa.size) - firstA[locA]
    M = int(cntA.max()) if pa.size else 0

    angq = np.zeros((n_own, nA, L), dtype=cdt)
    q4 = np.zeros((n_own, nA), dtype=cdt)
    # pair-force pieces that need p: store per-pair angular coefficient tensors
    fA_t1 = np.zeros((pa.size, nA, L), dtype=cdt)      # multiplies g'_n(j) u_j
    fA_t2 = np.zeros((pa.size, nA, L, 3), dtype=cdt)   # multiplies g_n(j)/r_j
    f4_a = np.zeros((pa.size, nA), dtype=cdt)          # multiplies g'_n(j) u_j
    f4_b = np.zeros((pa.size, nA, 3), dtype=cdt)       # multiplies 2 g_n(j)/r_j
    I3 = np.eye(3)
    for c0 in range(0, n_own, chunk):
        c1 = min(n_own, c0 + chunk)
        p0, p1 = firstA[c0], firstA[c1]
        if p1 == p0:
            continue
        nc = c1 - c0
        lo, sl = locA[p0:p1] - c0, slotA[p0:p1]
        G = np.zeros((nc, M, nA), dtype=cdt)
        U = np.zeros((nc, M, 3))
        G[lo, sl] = gA[p0:p1]
        U[lo, sl] = u[pa[p0:p1]]
        C = np.einsum("cja,cka->cjk", U, U)
        Pl, dPl = legendre(C, L)
        for l in range(1, L + 1):
            # q_nl = sum_jk g_n(j) g_n(k) P_l(c_jk)
            GP = np.einsum("ckn,cjk->cjn", G, Pl[l])          # sum_k G_kn P_l(c_jk)
            angq[c0:c1, :, l - 1] = np.einsum("cjn,cjn->cn", G, GP)
            fA_t1[p0:p1, :, l - 1] = 2.0 * GP[lo, sl]
            # sum_k G_kn P'_l(c_jk) (u_k - c_jk u_j)
            GdP = np.einsum("ckn,cjk->cjkn", G, dPl[l])
            v = np.einsum("cjkn,cka->cjna", GdP, U) - np.einsum("cjkn,cjk,cja->cjna", GdP, C, U)
            fA_t2[p0:p1, :, l - 1, :] = 2.0 * v[lo, sl]
        if h.has_4body:
            Mt = U[..., :, None] * U[..., None, :] - I3 / 3.0        # [c,M,3,3]
            Mt = Mt * (np.arange(M)[None, :] < cntA[c0:c1, None])[..., None, None]
            A = np.einsum("cjn,cjab->cnab", G, Mt)
            A2 = np.einsum("cnab,cnbd->cnad", A, A)
            q4[c0:c1] = np.einsum("cnab,cnba->cn", A2, A)
            # dq4/dr_j = 3[g' (u^T A^2 u - tr A^2/3) u + 2g/r (A^2 u - (u^T A^2 u) u)]
            uj = U[lo, sl]                                         # [p,3]
            A2j = A2[lo]                                           # [p,n,3,3]
            A2u = np.einsum("pnab,pb->pna", A2j, uj)
            uA2u = np.einsum("pa,pna->pn", uj, A2u)
            trA2 = np.einsum("pnaa->pn", A2j)
            f4_a[p0:p1] = 3.0 * (uA2u - trA2 / 3.0)
            f4_b[p0:p1] = 3.0 * (A2u - uA2u[..., None] * uj[:, None, :])
    o = h.n_rad
    q[:, o:o + nA * L] = angq.reshape(n_own, nA * L)
    if h.has_4body:
        q[:, o + nA * L:] = q4

    # network (Eq. 2, Section 2.3)
    tO = types[owners]
    W0, b0, w1, b1 = prm.W0[tO], prm.b0[tO], prm.w1[tO], prm.b1[tO]
    z = np.einsum("nhd,nd->nh", W0, q) + b0
    t = np.tanh(z)
    E = np.einsum("nh,nh->n", w1, t) + b1
    p = np.einsum("nh,nhd->nd", w1 * (1.0 - t * t), W0)

    # pair derivatives f_ij = dE_i/dr_ij
    f = (np.einsum("pn,pn->p", p[loc, :h.n_rad], dgR))[:, None] * u
    pang = p[:, o:o + nA * L].reshape(n_own, nA, L)[locA]        # [pa, n, l]
    fa = np.einsum("pnl,pn,pnl->p", pang, dgA, fA_t1)[:, None] * u[pa]
    fa = fa + np.einsum("pnl,pn,pnla->pa", pang, gA, fA_t2) / r[pa][:, None]
    if h.has_4body:
        p4 = p[:, o + nA * L:][locA]
        fa = fa + np.einsum("pn,pn,pn->p", p4, dgA, f4_a)[:, None] * u[pa]
        fa = fa + 2.0 * np.einsum("pn,pn,pna->pa", p4, gA, f4_b) / r[pa][:, None]
    f = f.astype(cdt)
    f[pa] += fa
    return q, E, p, f


def energy_forces_virial(h, theta, sys_pos, types, box, atom_off, pairs):
    """Whole-system E_i, F_i (Eq. 3) and per-config E_tot (Eq. 1) and V (Eq. 4).
    pairs = (i, j, s) with cutoff >= rc_rad (extra pairs are masked by r < rc)."""
    prm = unpack(h, theta)
    N = sys_pos.shape[0]
    i, j, s = pairs
    cfg = np.repeat(np.arange(box.shape[0]), np.diff(atom_off))
    rij = pair_vectors(sys_pos, box[cfg], i, j, s)
    owners = np.arange(N)
    q, E, p, f = atom_terms(h, prm, types, owners, i, j, rij)
    F = _segsum(f, i, N)
    np.subtract.at(F, j, f)
    B = box.shape[0]
    W = -f[:, :, None] * rij[:, None, :]                  # per pair -f (x) r
    V = np.zeros((B, 3, 3), dtype=f.dtype)
    np.add.at(V, cfg[i], W)
    Etot = np.zeros(B, dtype=E.dtype)
    np.add.at(Etot, cfg, E)
    return dict(q=q, E=E, p=p, F=F, Etot=Etot, V=V, f_pair=f, rij=rij)


def evaluate_centers(h, theta, pos32, pos64, types, box, atom_off, centers, skin_pairs_fn=None):
    """E_i, F_i and per-atom virial W_i = -sum_j f_ij (x) r_ij for a few centre
    atoms of a large system, from their neighbourhoods alone."""
    centers = np.unique(np.asarray(centers))
    i1, j1, _ = neighbor_pairs(pos32, box, atom_off, h.rc_rad, centers=centers)
    owners = np.unique(np.concatenate([centers, j1]))
    i, j, s = neighbor_pairs(pos32, box, atom_off, h.rc_rad, centers=owners)
    prm = unpack(h, theta)
    cfg = np.repeat(np.arange(box.shape[0]), np.diff(atom_off))
    rij = pair_vectors(pos64, box[cfg], i, j, s)
    q, E, p, f = atom_terms(h, prm, types, owners, i, j, rij)
    loc_c = np.searchsorted(owners, centers)
    Fc = np.zeros((centers.size, 3), dtype=f.dtype)
    Wc = np.zeros((centers.size, 3, 3), dtype=f.dtype)
    ci = np.searchsorted(centers, i)
    ok_i = (ci < centers.size) & (centers[np.minimum(ci, centers.size - 1)] == i)
    np.add.at(Fc, ci[ok_i], f[ok_i])
    np.add.at(Wc, ci[ok_i], -f[ok_i][:, :, None] * rij[ok_i][:, None, :])
    cj = np.searchsorted(centers, j)
    ok_j = (cj < centers.size) & (centers[np.minimum(cj, centers.size - 1)] == j)
    np.subtract.at(Fc, cj[ok_j], f[ok_j])
    return dict(centers=centers, E=E[loc_c], q=q[loc_c], F=Fc, W=Wc)


# ---------------------------------------------------------------------------
# loss (Eqs. 18-21) and its parameter gradient
# ---------------------------------------------------------------------------
def loss_value(h, theta, pos, types, box, atom_off, pairs, E_lbl, F_lbl, V_lbl,
               w=(1.0, 1.0, 0.1), mode=0):
    """mode 0: L = 1/B sum_b [wE (dE_b/N_b)^2 + wF/(3N_b) sum dF^2 + wV/9 sum (dV_b/N_b)^2]
    mode 1: L = 1/B sum_b [wE/N_b dE_b^2 + wF/(3N_b) sum dF^2 + wV/(9N_b) sum dV_b^2]
    (Eqs. 19-21 per configuration, averaged over the batch).  A configuration
    with N_b = 0 adds no term but counts in B (the paper is silent there)."""
    out = energy_forces_virial(h, theta, pos, types, box, atom_off, pairs)
    Nb = np.diff(atom_off).astype(np.float64)
    B = Nb.size
    cfg = np.repeat(np.arange(B), np.diff(atom_off))
    dE = out["Etot"] - E_lbl
    dF = out["F"] - F_lbl
    dV = (out["V"] - V_lbl.reshape(B, 3, 3)).reshape(B, 9)
    sF = np.zeros(B, dtype=dF.dtype)
    np.add.at(sF, cfg, (dF * dF).sum(1))
    # a configuration with no atoms has no per-atom normalisation: it adds no
    # term but still counts in B
    has = Nb > 0
    n = np.where(has, Nb, 1.0)
    if mode == 0:
        Lb = w[0] * (dE / n) ** 2 + w[1] * sF / (3 * n) + w[2] * ((dV / n[:, None]) ** 2).sum(1) / 9.0
    elif mode == 1:
        Lb = w[0] * dE ** 2 / n + w[1] * sF / (3 * n) + w[2] * (dV ** 2).sum(1) / (9.0 * n)
    else:
        raise ValueError(mode)
    return np.where(has, Lb, 0.0).sum() / B


def adjoint_functional(h, theta, pos, types, box, atom_off, pairs, aE, lamF, muV):
    """Phi = sum_b aE_b E_b + sum_i lamF_i . F_i + sum_b muV_b : V_b."""
    out = energy_forces_virial(h, theta, pos, types, box, atom_off, pairs)
    B = box.shape[0]
    return ((aE * out["Etot"]).sum() + (lamF * out["F"]).sum()
            + (muV.reshape(B, 3, 3) * out["V"]).sum())


def complex_step_grad(fun, theta, indices, h_step=1e-30):
    """d fun / d theta_k for k in indices: Im fun(theta + i h e_k) / h."""
    g = np.zeros(len(indices))
    for a, k in enumerate(indices):
        th = theta.astype(np.complex128)
        th[k] += 1j * h_step
        g[a] = np.imag(fun(th)) / h_step
    return g


# ---------------------------------------------------------------------------
# molecular dynamics: velocity Verlet around the forces of Eq. 3
# ---------------------------------------------------------------------------
# 1 u A^2 / fs^2 expressed in eV, from the CODATA atomic mass constant and the
# elementary charge: a = F / (m * MVV_EV) in A/fs^2 for F in eV/A and m in u.
ATOMIC_MASS_KG = 1.66053906660e-27
ELEMENTARY_CHARGE_C = 1.602176634e-19
MVV_EV = ATOMIC_MASS_KG * 1e-20 / 1e-30 / ELEMENTARY_CHARGE_C


def wrap_positions(pos, box, atom_off):
    """Each atom's coordinates mapped into [0, L) of its configuration's box."""
    cfg = np.repeat(np.arange(box.shape[0]), np.diff(atom_off))
    L = box[cfg]
    return pos - L * np.floor(pos / L)


def kinetic_energy(vel, types, masses, atom_off):
    """Per-configuration sum of m v^2 / 2 in eV (v in A/fs, m in u)."""
    B = len(atom_off) - 1
    cfg = np.repeat(np.arange(B), np.diff(atom_off))
    ke = 0.5 * MVV_EV * np.asarray(masses, np.float64)[types] * (vel * vel).sum(1)
    out = np.zeros(B)
    np.add.at(out, cfg, ke)
    return out


def velocity_verlet(h, theta, pos, vel, types, box, atom_off, masses, dt, n_steps, rebuild_every=10,
                    force=None):
    """n_steps of velocity Verlet in FP64, each step in this order:
    v += dt/2 F/(m MVV_EV); x += dt v; at every rebuild_every-th step
    (counting from step 0) x is wrapped into the box; F = F(x) by Eq. 3 over
    every pair inside rc_rad at the new positions; v += dt/2 F/(m MVV_EV).
    force: F at the starting positions (evaluated here when None).
    Returns the final pos, vel and F, and per step the potential and
    kinetic energy of every configuration."""
    pos = np.array(pos, np.float64)
    vel = np.array(vel, np.float64)
    types = np.asarray(types)
    inv_m = 1.0 / (np.asarray(masses, np.float64)[types] * MVV_EV)

    def forces(x):
        pairs = neighbor_pairs(x.astype(np.float32), box, atom_off, h.rc_rad)
        out = energy_forces_virial(h, theta, x, types, box, atom_off, pairs)
        return out["F"], out["Etot"]

    F = np.array(force, np.float64) if force is not None else forces(pos)[0]
    epot, ekin = [], []
    for k in range(n_steps):
        vel = vel + 0.5 * dt * F * inv_m[:, None]
        pos = pos + dt * vel
        if k % rebuild_every == 0:
            pos = wrap_positions(pos, box, atom_off)
        F, E = forces(pos)
        vel = vel + 0.5 * dt * F * inv_m[:, None]
        epot.append(E)
        ekin.append(kinetic_energy(vel, types, masses, atom_off))
    return dict(pos=pos, vel=vel, F=F, epot=np.array(epot), ekin=np.array(ekin))


# ---------------------------------------------------------------------------
# optimiser (Section 3.3.1)
# ---------------------------------------------------------------------------
def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Section 3.3.1, no weight decay), in FP64: the moving
    averages m and v of g and g^2, their bias-corrected values m/(1-beta1^t)
    and v/(1-beta2^t), and the step lr * mhat / (sqrt(vhat) + eps).
    Returns (theta, m, v) after step t (t = 1 for the first step)."""
    theta = np.asarray(theta, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v

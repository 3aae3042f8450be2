"""Seeded synthetic Ge-Sb-Te-shaped inputs for the NEP path.

This module is the only code shared by the CUDA path's tests/bench and the
FP64 oracle.  It holds no NEP arithmetic: it draws structures (rock-salt
lattices with cation vacancies, random sequential-adsorption packings),
species, parameter vectors and Maxwell-Boltzmann velocities, all from
counter-free NumPy PCG64 streams keyed by (seed, tag).

Seeds: 0 structures, 1 weights, 2 teacher weights, 3 velocities.
Species indices: 0 = Ge, 1 = Sb, 2 = Te.  Units: Angstrom, u, fs.

The paper's Ge-Sb-Te dataset (Section 4.1) is not available; these seeded
structures stand in for it with the same composition, density and
neighbour statistics.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASSES = np.array([72.63, 121.76, 127.60])  # Ge, Sb, Te in u
KB_EV = 8.617333262e-5                       # Boltzmann constant, eV/K
MVV_TO_EV = 103.6427                         # 1 u*A^2/fs^2 in eV

SEED_STRUCT, SEED_WEIGHTS, SEED_TEACHER, SEED_VEL = 0, 1, 2, 3


def rng_for(seed: int, *tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, *tag]))


# --------------------------------------------------------------------------
# hyper-parameters (the NEP model shape; Section 2.3 and Table 2)
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Hyper:
    n_types: int = 3
    n_rad: int = 8       # radial descriptor count (n = 0..n_rad-1)
    n_ang: int = 6       # angular n count
    k_rad: int = 8       # Chebyshev basis functions, radial
    k_ang: int = 8       # Chebyshev basis functions, angular
    l_max: int = 4
    has_4body: int = 1
    n_hidden: int = 30
    rc_rad: float = 7.0
    rc_ang: float = 5.0

    @property
    def dim(self) -> int:
        return self.n_rad + self.n_ang * self.l_max + (self.n_ang if self.has_4body else 0)

    @property
    def n_mlp(self) -> int:
        return self.n_types * (self.n_hidden * self.dim + 2 * self.n_hidden + 1)

    @property
    def n_c(self) -> int:
        t2 = self.n_types * self.n_types
        return t2 * (self.n_rad * self.k_rad + self.n_ang * self.k_ang)

    @property
    def n_params(self) -> int:
        return self.n_mlp + self.n_c


# 216-atom config: 38-dim descriptor, MLP 38->30->1
HYPER_SMALL = Hyper()
# 3.7M-atom config: n_R=12, n_A=8, l_max=4 + 4-body, MLP ->64
HYPER_LARGE = Hyper(n_rad=12, n_ang=8, n_hidden=64)
# the paper's own Table 2 model: 2+3-body only, 50 neurons
HYPER_TABLE2 = Hyper(n_rad=10, n_ang=8, has_4body=0, n_hidden=50)


def init_params(h: Hyper, seed: int = SEED_WEIGHTS) -> np.ndarray:
    """Flat float64 parameter vector in the library's order:
    for t in types: W0[t][H][D], b0[t][H], w1[t][H], b1[t];
    then cR[Zi][Zj][n_rad][k_rad]; then cA[Zi][Zj][n_ang][k_ang].
    W0, b0 ~ U(+-1/sqrt(D)); w1, b1 ~ U(+-1/sqrt(H)); c ~ N(0, 0.1^2)."""
    rng = rng_for(seed, 1000)
    D, H, T = h.dim, h.n_hidden, h.n_types
    parts = []
    for _ in range(T):
        a = 1.0 / math.sqrt(D)
        b = 1.0 / math.sqrt(H)
        parts.append(rng.uniform(-a, a, size=H * D))
        parts.append(rng.uniform(-a, a, size=H))
        parts.append(rng.uniform(-b, b, size=H))
        parts.append(rng.uniform(-b, b, size=1))
    parts.append(rng.normal(0.0, 0.1, size=T * T * h.n_rad * h.k_rad))
    parts.append(rng.normal(0.0, 0.1, size=T * T * h.n_ang * h.k_ang))
    theta = np.concatenate(parts)
    assert theta.size == h.n_params
    return theta


# --------------------------------------------------------------------------
# structures
# --------------------------------------------------------------------------
@dataclass
class System:
    """A batch of B periodic orthorhombic configurations, atoms concatenated."""
    pos: np.ndarray            # [N, 3] float64, wrapped into [0, L)
    types: np.ndarray          # [N] int32
    box: np.ndarray            # [B, 3] float64
    atom_off: np.ndarray       # [B+1] int64 CSR offsets
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_cfg(self) -> int:
        return int(self.box.shape[0])

    def cfg_of_atom(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_cfg), np.diff(self.atom_off))

    def pos32(self) -> np.ndarray:
        """Float32 positions as the GPU path stores them, wrapped into [0, L)."""
        box32 = self.box.astype(np.float32)[self.cfg_of_atom()]
        p = self.pos.astype(np.float32)
        p = np.where(p >= box32, p - box32, p)
        p = np.where(p < 0, p + box32, p)
        p = np.where(p >= box32, np.float32(0), p)
        return p.astype(np.float32)


def _wrap(pos: np.ndarray, L: np.ndarray) -> np.ndarray:
    p = pos - np.floor(pos / L) * L
    return np.where(p >= L, p - L, p)


def rocksalt(ncell: int, a: float = 6.0, vacancy: float = 0.0, ge_frac_of_cations: float = 0.5,
             jitter: float = 0.1, seed: int = SEED_STRUCT, tag: int = 0) -> System:
    """ncell^3 conventional rock-salt cells (8 sites each), Te on the anion
    sublattice, cation sites shuffled to exact Ge/Sb/vacancy counts, Gaussian
    jitter.  vacancy is the vacant fraction of cation sites; the remaining
    cations split Ge/Sb 1:1."""
    rng = rng_for(seed, 10 + tag)
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    anion = fcc + np.array([.5, 0, 0])
    g = np.arange(ncell)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    cat = (cells[:, None, :] + fcc[None]).reshape(-1, 3) * a
    ani = (cells[:, None, :] + anion[None]).reshape(-1, 3) * a
    n_cat = cat.shape[0]
    n_vac = int(round(vacancy * n_cat))
    n_ge = (n_cat - n_vac) // 2
    n_sb = n_cat - n_vac - n_ge
    lab = np.concatenate([np.zeros(n_ge, np.int32), np.ones(n_sb, np.int32),
                          np.full(n_vac, -1, np.int32)])
    rng.shuffle(lab)
    keep = lab >= 0
    # interleave cations and anions cell by cell so that index order follows space
    pos = np.concatenate([cat[keep], ani])
    types = np.concatenate([lab[keep], np.full(ani.shape[0], 2, np.int32)])
    cell_id = np.concatenate([np.repeat(np.arange(cells.shape[0]), 4)[keep],
                              np.repeat(np.arange(cells.shape[0]), 4)])
    order = np.argsort(cell_id, kind="stable")
    pos, types = pos[order], types[order]
    pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    L = np.full(3, ncell * a)
    pos = _wrap(pos, L)
    return System(pos=pos, types=types.astype(np.int32), box=L[None, :].copy(),
                  atom_off=np.array([0, pos.shape[0]], np.int64),
                  meta=dict(kind="rocksalt", ncell=ncell, a=a, vacancy=vacancy))


def rsa_pack(rng: np.random.Generator, n: int, L: float, dmin: float) -> np.ndarray:
    """Random sequential adsorption in a periodic cube: uniform candidates are
    accepted in draw order when no accepted point lies within dmin."""
    from scipy.spatial import cKDTree
    acc = np.empty((0, 3))
    while acc.shape[0] < n:
        k = max(64, 2 * (n - acc.shape[0]))
        cand = rng.uniform(0.0, L, size=(k, 3))
        cand = np.where(cand >= L, 0.0, cand)
        if acc.shape[0]:
            d, _ = cKDTree(acc, boxsize=L).query(cand, k=1)
            cand = cand[d >= dmin]
        if cand.shape[0] == 0:
            continue
        pairs = cKDTree(cand, boxsize=L).query_pairs(dmin, output_type="ndarray")
        ok = np.ones(cand.shape[0], bool)
        if pairs.size:
            later = {}
            for a_, b_ in pairs:
                lo, hi = (a_, b_) if a_ < b_ else (b_, a_)
                later.setdefault(hi, []).append(lo)
            for hi in sorted(later):
                if any(ok[lo] for lo in later[hi]):
                    ok[hi] = False
        acc = np.concatenate([acc, cand[ok]])
    return acc[:n]


def packing_batch(counts, density: float = 0.0325, dmin: float = 2.4,
                  seed: int = SEED_STRUCT, tag: int = 0) -> System:
    """Batch of cubic periodic random packings, one per entry of counts,
    L = (N/density)^(1/3), Ge:Sb:Te = 2:2:5 (n_Ge = n_Sb = round(2N/9))."""
    pos_l, typ_l, box_l = [], [], []
    for b, n in enumerate(counts):
        rng = rng_for(seed, 20 + tag, b)
        L = (n / density) ** (1.0 / 3.0)
        p = rsa_pack(rng, int(n), L, dmin)
        n_ge = int(round(2 * n / 9))
        t = np.concatenate([np.zeros(n_ge, np.int32), np.ones(n_ge, np.int32),
                            np.full(n - 2 * n_ge, 2, np.int32)])
        rng.shuffle(t)
        pos_l.append(p)
        typ_l.append(t)
        box_l.append([L, L, L])
    counts = np.asarray(counts, np.int64)
    return System(pos=np.concatenate(pos_l), types=np.concatenate(typ_l),
                  box=np.array(box_l, np.float64),
                  atom_off=np.concatenate([[0], np.cumsum(counts)]).astype(np.int64),
                  meta=dict(kind="packing", density=density, dmin=dmin))


def uniform_counts(n_cfg: int, lo: int, hi: int, seed: int = SEED_STRUCT, tag: int = 0) -> np.ndarray:
    return rng_for(seed, 30 + tag).integers(lo, hi + 1, size=n_cfg)


def loguniform_counts(n_cfg: int, lo: int, hi: int, seed: int = SEED_STRUCT, tag: int = 0) -> np.ndarray:
    u = rng_for(seed, 40 + tag).uniform(math.log(lo), math.log(hi), size=n_cfg)
    return np.clip(np.round(np.exp(u)).astype(np.int64), lo, hi)


def maxwell_boltzmann(types: np.ndarray, temp: float = 900.0, seed: int = SEED_VEL,
                      atom_off: np.ndarray | None = None) -> np.ndarray:
    """Velocities in A/fs: sigma = sqrt(kB T / (m * 103.6427)) per component,
    centre-of-mass velocity removed per configuration."""
    rng = rng_for(seed, 50)
    m = MASSES[types]
    sig = np.sqrt(KB_EV * temp / (m * MVV_TO_EV))
    v = rng.normal(size=(types.size, 3)) * sig[:, None]
    off = atom_off if atom_off is not None else np.array([0, types.size])
    for b in range(len(off) - 1):
        s = slice(off[b], off[b + 1])
        mm = m[s]
        if mm.size:                                # an empty configuration has no centre of mass
            v[s] -= (mm[:, None] * v[s]).sum(0) / mm.sum()
    return v


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def workload_cell216() -> tuple[System, Hyper]:
    """216 atoms: 3^3 rock-salt cells, a = 6 A, Ge/Sb 1:1 on cations."""
    return rocksalt(3, vacancy=0.0, tag=0), HYPER_SMALL


def workload_md900k() -> tuple[System, Hyper]:
    """900,000 atoms: 50^3 cells, 20% cation vacancies (config of the MD bench)."""
    return rocksalt(50, vacancy=0.2, tag=1), HYPER_SMALL


def workload_train128() -> tuple[System, Hyper]:
    """128 packings, N ~ U{24..512}."""
    return packing_batch(uniform_counts(128, 24, 512, tag=2), tag=2), HYPER_SMALL


def workload_mixed3m7() -> tuple[System, Hyper]:
    """3,686,400 atoms: 80^3 cells, 20% cation vacancies, larger NEP."""
    return rocksalt(80, vacancy=0.2, tag=3), HYPER_LARGE


def workload_replicas1024() -> tuple[System, Hyper]:
    """1,024 packings, N log-uniform in [64, 4096]."""
    return packing_batch(loguniform_counts(1024, 64, 4096, tag=4), tag=4), HYPER_SMALL

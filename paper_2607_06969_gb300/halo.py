"""Molecular dynamics of one large periodic system over several GPUs with a
point-to-point ghost halo: slabs along x, one rank per GPU, each rank keeping
only its own atoms (the paper runs LAMMPS with one MPI domain per device,
Section 3.5; this is that decomposition for the NEP path).

Rank r owns the atoms with x in its slab [lo, hi).  Its local system is
[own atoms | ghosts from the left neighbour | ghosts from the right
neighbour] in a frame whose x starts at lo - halo.  With halo = 2 (rc + skin)
the ghosts hold every neighbour of an owned atom and those neighbours' own
neighbourhoods, so the owned atoms' forces, energies and virials are those of
the whole-system evaluation and nothing flows back from the ghosts.

Every step:
  * half kick and drift of the own atoms (nep_md_kick);
  * at a rebuild step (every `rebuild_every` steps): atoms that left the slab
    move to the neighbour with their velocities, species and ids; the own
    atoms within `halo` of each face are chosen as the ghosts that face's
    neighbour receives until the next rebuild, and the ghosts' species are
    exchanged;
  * ghost positions go to the two neighbours (one message each way per face)
    and the local system is assembled (nep_domain_take / nep_domain_place);
  * the local list is rebuilt at a rebuild step; the owned atoms are
    evaluated (nep_energy_forces_virial_owned);
  * half kick of the own atoms.
Per step a rank sends and receives the positions of the atoms in two bands of
width `halo`: 2 x rho x halo x L_y x L_z x 12 bytes each way, whatever the
number of ranks (1.15 MB for the 900k-atom, 300 A box).  Energies and virials
stay per rank until `totals` sums them (one all-reduce of 10 doubles).

The step is written once as a generator that yields each exchange it needs
(`Exchange`: a ring shift of a few tensors).  `run_dist` serves the
exchanges with torch.distributed point-to-point calls (NCCL between GPUs);
`run_emulated` serves the exchanges of all ranks of one process in lockstep,
which lets one GPU (or the CPU) run a whole decomposition rank after rank
with no kernel of one rank waiting on another's.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as nb


class Exchange:
    """A ring shift: send `tensors` (each [ncomp][n], n may differ per rank)
    to rank (r + d) mod world and receive the same list from rank
    (r - d) mod world.  `recv_cols`, when the receiver already knows them,
    are the column counts it will receive (no count exchange is needed)."""

    def __init__(self, d: int, tensors, recv_cols=None):
        self.d, self.tensors = d, list(tensors)
        self.recv_cols = None if recv_cols is None else list(recv_cols)


def plan(Lx: float, world: int, rc: float, skin: float) -> tuple[list[tuple[float, float]], float]:
    """Equal slabs [lo, hi) of [0, Lx) and the halo 2 (rc + skin).  Every
    slab must be at least one halo wide, so that a face's ghosts all belong
    to the rank across that face."""
    if world < 2:
        raise ValueError("a slab decomposition needs at least two ranks (one rank runs the whole system)")
    halo = 2.0 * (rc + skin)
    w = Lx / world
    if w < halo:
        raise ValueError(f"{world} slabs of {w:.2f} A are narrower than the halo of {halo:.2f} A")
    edges = [Lx * r / world for r in range(world + 1)]
    return [(float(edges[r]), float(edges[r + 1])) for r in range(world)], halo


class LibOps:
    """The device operations of a rank, through libnep (one GPU)."""

    def __init__(self, model: nb.Model, device="cuda"):
        import torch
        self.model, self.device, self.torch = model, device, torch
        self._band_work = None

    def empty(self, shape, dtype):
        return self.torch.empty(shape, dtype=dtype, device=self.device)

    def band(self, pos, n: int, lo: float, hi: float):
        """Indices (ascending) of the first n atoms of pos [3][n] with x in [lo, hi)."""
        torch = self.torch
        need = int(nb.lib().nep_domain_workspace_bytes(n))
        if self._band_work is None or self._band_work.numel() < need + 256:
            self._band_work = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        w = ctypes.c_void_p(self._band_work.data_ptr() + (-self._band_work.data_ptr()) % 256)
        idx = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        counts = torch.zeros(2, dtype=torch.int32, device=self.device)
        nb.check(nb.lib().nep_domain_band(nb._ptr(pos), n, ctypes.c_float(lo), ctypes.c_float(hi), nb._ptr(idx),
                                          n, nb._ptr(counts), w, need, nb._stream()), "nep_domain_band")
        return idx[:int(counts[0].item())]

    def take(self, src, n_src: int, idx):
        """src [c][n_src] at columns idx -> [c][len(idx)]."""
        c = src.shape[0]
        out = self.empty((c, max(idx.numel(), 1)), src.dtype)[:, :idx.numel()]
        nb.check(nb.lib().nep_domain_take(nb._ptr(src), n_src, c, nb._ptr(idx), idx.numel(), nb._ptr(out),
                                          nb._stream()), "nep_domain_take")
        return out

    def place(self, src, n: int, box_x: float, x_center: float, x_origin: float, dst, stride: int, offset: int):
        """dst[c][offset + l] = src[c][l] (row stride `stride`), x brought to
        the image nearest x_center and taken relative to x_origin when box_x > 0."""
        nb.check(nb.lib().nep_domain_place(nb._ptr(src), n, src.shape[0], ctypes.c_float(box_x),
                                           ctypes.c_float(x_center), ctypes.c_float(x_origin), nb._ptr(dst),
                                           stride, offset, nb._stream()), "nep_domain_place")

    def kick(self, sys_, vel, force, masses, half_dt: float, drift_dt: float):
        nb.check(nb.lib().nep_md_kick(self.model.handle, ctypes.byref(sys_.c), nb._ptr(vel), nb._ptr(force),
                                      masses.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(half_dt),
                                      ctypes.c_float(drift_dt), nb._stream()), "nep_md_kick")

    def wrap(self, sys_):
        """Every coordinate of sys_'s atoms into [0, L) of its box (nep_md_wrap)."""
        nb.check(nb.lib().nep_md_wrap(self.model.handle, ctypes.byref(sys_.c), nb._stream()), "nep_md_wrap")

    def neighbors(self, loc, nl, skin: float, ws):
        nb.neighbors(self.model, loc, nl, skin, ws)

    def evaluate_owned(self, loc, nl, n_owned: int, force, e_tot, vir, ws):
        nb.check(nb.lib().nep_energy_forces_virial_owned(
            self.model.handle, ctypes.byref(loc.c), ctypes.byref(nl.c), n_owned, None, nb._ptr(force),
            nb._ptr(e_tot), nb._ptr(vir), ws.ptr, ws.bytes, nb._stream()), "nep_energy_forces_virial_owned")

    def workspace(self, n_atoms: int, cap: int, cap_ang: int):
        return nb.Workspace(self.model, n_atoms, 1, cap, cap_ang, device=self.device)

    def check_list(self, nl) -> None:
        st = nb.check_list(nl)
        if st != nb.NEP_OK:
            raise nb.NepError(st, "local neighbour list", nb.last_error())


class SlabRank:
    """One rank of the decomposition.  `box` is the whole system's edges
    (orthorhombic), `masses` one per species (u), dt in fs."""

    def __init__(self, ops, rank: int, world: int, box, lo: float, hi: float, halo: float, skin: float,
                 masses, dt: float = 2.0, rebuild_every: int = 10, cap: int = 112, cap_ang: int = 56,
                 rc: float = 7.0):
        from .spatial import LocalList, LocalSystem
        self._LocalList, self._LocalSystem = LocalList, LocalSystem
        self.ops, self.rank, self.world = ops, rank, world
        self.box = np.asarray(box, np.float64).reshape(3)
        self.lo, self.hi, self.halo, self.skin = float(lo), float(hi), float(halo), float(skin)
        self.masses = np.ascontiguousarray(np.asarray(masses, np.float32))
        self.dt, self.every = float(dt), int(rebuild_every)
        self.cap, self.cap_ang = cap, cap_ang
        self.origin = self.lo - self.halo
        self.center = 0.5 * (self.lo + self.hi)
        pad = rc + skin + 1.0
        self.box_local = np.array([self.hi - self.lo + 2.0 * self.halo + pad, self.box[1], self.box[2]],
                                  np.float32)
        self.k = 0
        self.n_own = 0
        self.loc = None

    # ----------------------------------------------------------------- state
    def load(self, pos, types, vel, gid=None) -> None:
        """Take this rank's atoms (x in [lo, hi), decided in FP32) from the
        whole system's host arrays pos [N,3], types [N], vel [N,3]."""
        torch = self.ops.torch
        pos = np.asarray(pos, np.float32)
        x = pos[:, 0]
        own = np.nonzero((x >= np.float32(self.lo)) & (x < np.float32(self.hi)))[0]
        gid = np.arange(pos.shape[0], dtype=np.int32) if gid is None else np.asarray(gid, np.int32)
        dev = self.ops.device
        self._set_own(torch.from_numpy(np.ascontiguousarray(pos[own].T)).to(dev),
                      torch.from_numpy(np.ascontiguousarray(np.asarray(vel, np.float32)[own].T)).to(dev),
                      torch.from_numpy(np.ascontiguousarray(np.asarray(types, np.int32)[own][None, :])).to(dev),
                      torch.from_numpy(np.ascontiguousarray(gid[own][None, :])).to(dev))

    def _set_own(self, pos, vel, typ, gid) -> None:
        """Own arrays, contiguous [c][n_own]; the kick sees them as one
        configuration of n_own atoms."""
        torch = self.ops.torch
        n = pos.shape[1]
        self.n_own = n
        self.pos, self.vel = pos.contiguous(), vel.contiguous()
        self.typ, self.gid = typ.contiguous(), gid.contiguous()
        self.force = torch.zeros_like(self.pos)
        self.own_sys = self._LocalSystem(max(n, 1), self.box, self.ops.device)
        self.own_sys.pos_buf = self.pos.reshape(-1) if n > 0 else self.own_sys.pos_buf
        self.own_sys.type = self.typ.reshape(-1) if n > 0 else self.own_sys.type
        self.own_sys.resize(n)
        self.arange = torch.arange(max(n, 1), dtype=torch.int32, device=self.ops.device)

    # ----------------------------------------------------------- exchanges
    def _rebuild(self):
        """Migration of the atoms that left the slab, then the ghost plan."""
        torch, ops = self.ops.torch, self.ops
        n = self.n_own
        inf = float("inf")
        parts = []
        for lo, hi in ((-inf, self.lo), (self.hi, inf), (self.lo, self.hi)):
            idx = ops.band(self.pos, n, lo, hi)
            parts.append([ops.take(t, n, idx) for t in (self.pos, self.vel, self.typ, self.gid)])
        to_left, to_right, stay = parts
        from_right = yield Exchange(-1, to_left)
        from_left = yield Exchange(+1, to_right)
        groups = [stay, from_left, from_right]
        m = sum(g[0].shape[1] for g in groups)
        pos = ops.empty((3, max(m, 1)), torch.float32)[:, :m]
        vel = ops.empty((3, max(m, 1)), torch.float32)[:, :m]
        typ = ops.empty((1, max(m, 1)), torch.int32)[:, :m]
        gid = ops.empty((1, max(m, 1)), torch.int32)[:, :m]
        off = 0
        for g in groups:
            c = g[0].shape[1]
            ops.place(g[0], c, float(self.box[0]), self.center, 0.0, pos, m, off)
            ops.place(g[1], c, 0.0, 0.0, 0.0, vel, m, off)
            ops.place(g[2], c, 0.0, 0.0, 0.0, typ, m, off)
            ops.place(g[3], c, 0.0, 0.0, 0.0, gid, m, off)
            off += c
        self._set_own(pos, vel, typ, gid)
        # every own atom now lies in [lo, hi) in x; y and z, which drift
        # freely between rebuilds, go back into the box (x stays as it is)
        ops.wrap(self.own_sys)
        # ghosts: the own atoms within halo of each face, fixed until the next rebuild
        self.idx_to_left = ops.band(self.pos, self.n_own, self.lo, self.lo + self.halo)
        self.idx_to_right = ops.band(self.pos, self.n_own, self.hi - self.halo, self.hi)
        (t_from_right,) = yield Exchange(-1, [ops.take(self.typ, self.n_own, self.idx_to_left)])
        (t_from_left,) = yield Exchange(+1, [ops.take(self.typ, self.n_own, self.idx_to_right)])
        self.n_gl, self.n_gr = t_from_left.shape[1], t_from_right.shape[1]
        self.n_local = self.n_own + self.n_gl + self.n_gr
        nl_ = self.n_local
        if self.loc is None or nl_ > self.loc.cap:
            cap_atoms = int(1.25 * nl_) + 256
            self.loc = self._LocalSystem(cap_atoms, self.box_local, ops.device)
            self.nl = self._LocalList(cap_atoms, self.cap, self.cap_ang, ops.device)
            self.ws = ops.workspace(cap_atoms, self.cap, self.cap_ang)
            self.force_buf = torch.zeros(3 * cap_atoms, dtype=torch.float32, device=ops.device)
            self.e_tot = torch.zeros(1, dtype=torch.float64, device=ops.device)
            self.vir = torch.zeros(1, 9, dtype=torch.float64, device=ops.device)
        self.loc.resize(nl_)
        self.nl.resize(nl_)
        self.force_local = self.force_buf[:3 * max(nl_, 1)].view(3, max(nl_, 1))
        ltype = self.loc.type.view(1, -1)
        ops.place(self.typ, self.n_own, 0.0, 0.0, 0.0, ltype, nl_, 0)
        ops.place(t_from_left, self.n_gl, 0.0, 0.0, 0.0, ltype, nl_, self.n_own)
        ops.place(t_from_right, self.n_gr, 0.0, 0.0, 0.0, ltype, nl_, self.n_own + self.n_gl)
        self.need_list = True

    def _forces(self):
        """Ghost positions in, local system assembled, owned atoms evaluated."""
        ops = self.ops
        n, nl_ = self.n_own, self.n_local
        lpos = self.loc.pos
        Lx = float(self.box[0])
        ops.place(self.pos, n, Lx, self.center, self.origin, lpos, nl_, 0)
        (p_from_right,) = yield Exchange(-1, [ops.take(self.pos, n, self.idx_to_left)], [self.n_gr])
        (p_from_left,) = yield Exchange(+1, [ops.take(self.pos, n, self.idx_to_right)], [self.n_gl])
        ops.place(p_from_left, self.n_gl, Lx, self.lo - 0.5 * self.halo, self.origin, lpos, nl_, n)
        ops.place(p_from_right, self.n_gr, Lx, self.hi + 0.5 * self.halo, self.origin, lpos, nl_, n + self.n_gl)
        if self.need_list:
            ops.neighbors(self.loc, self.nl, self.skin, self.ws)
            self.need_list = False
        ops.evaluate_owned(self.loc, self.nl, n, self.force_local, self.e_tot, self.vir, self.ws)
        self.force = ops.take(self.force_local, nl_, self.arange[:n])

    # ------------------------------------------------------------ the steps
    def start(self):
        """Generator: the first ghost plan, list and forces."""
        yield from self._rebuild()
        yield from self._forces()

    def step(self):
        """Generator: one velocity-Verlet step."""
        self.ops.kick(self.own_sys, self.vel, self.force, self.masses, 0.5 * self.dt, self.dt)
        self.k += 1
        if self.k % self.every == 0:
            yield from self._rebuild()
        yield from self._forces()
        self.ops.kick(self.own_sys, self.vel, self.force, self.masses, 0.5 * self.dt, 0.0)

    def check(self) -> None:
        self.ops.check_list(self.nl)


# ---------------------------------------------------------------- runners
def run_emulated(gens) -> None:
    """Drive one generator per rank of a decomposition held in this process:
    all ranks advance to their next exchange, then the exchange is served
    (rank r receives what rank r - d sent), in lockstep until they finish."""
    world = len(gens)
    reqs = []
    for g in gens:
        try:
            reqs.append(next(g))
        except StopIteration:
            reqs.append(None)
    while any(r is not None for r in reqs):
        if any(r is None for r in reqs):
            raise RuntimeError("ranks disagree on the number of exchanges")
        d = reqs[0].d
        if any(r.d != d for r in reqs):
            raise RuntimeError("ranks disagree on the direction of an exchange")
        recv = [reqs[(r - d) % world].tensors for r in range(world)]
        for r in range(world):
            if reqs[r].recv_cols is not None and [t.shape[1] for t in recv[r]] != reqs[r].recv_cols:
                raise RuntimeError("a rank received other column counts than it expected")
        for r, g in enumerate(gens):
            try:
                reqs[r] = g.send(recv[r])
            except StopIteration:
                reqs[r] = None


def dist_shift(dist, d: int, tensors, rank: int, world: int, recv_cols=None, host_staging: bool = False):
    """One ring shift with torch.distributed point-to-point calls: the column
    counts first (unless the receiver knows them), then the data (empty
    transfers skipped on both sides).  host_staging: the data travel through
    host memory (a backend without device transfers, such as gloo)."""
    import torch
    to, frm = (rank + d) % world, (rank - d) % world
    dev_out = tensors[0].device
    if host_staging:
        tensors = [t.cpu() for t in tensors]
    dev = tensors[0].device
    if recv_cols is None:
        sizes = torch.tensor([t.shape[1] for t in tensors], dtype=torch.int64, device=dev)
        rsizes = torch.empty_like(sizes)
        for w in dist.batch_isend_irecv([dist.P2POp(dist.isend, sizes, to),
                                         dist.P2POp(dist.irecv, rsizes, frm)]):
            w.wait()
        rs = rsizes.tolist()
    else:
        rs = list(recv_cols)
    out = [torch.empty((t.shape[0], rs[k]), dtype=t.dtype, device=dev) for k, t in enumerate(tensors)]
    ops = []
    for k, t in enumerate(tensors):
        if t.shape[1] > 0:
            ops.append(dist.P2POp(dist.isend, t.contiguous(), to))
        if rs[k] > 0:
            ops.append(dist.P2POp(dist.irecv, out[k], frm))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()
    return [t.to(dev_out) for t in out] if host_staging else out


def run_dist(gen, dist, rank: int, world: int, host_staging: bool = False) -> None:
    """Drive this process's rank generator, serving its exchanges with the
    process group (one rank per process)."""
    try:
        req = next(gen)
        while True:
            req = gen.send(dist_shift(dist, req.d, req.tensors, rank, world, req.recv_cols, host_staging))
    except StopIteration:
        pass


def totals(ranks_or_rank, dist=None):
    """Whole-system energy [1] and virial [1, 9]: the sum of the ranks' owned
    sums (in-process ranks summed here, or one all-reduce over the group)."""
    import torch
    if dist is None:
        e = sum(r.e_tot.double().cpu() for r in ranks_or_rank)
        v = sum(r.vir.double().cpu() for r in ranks_or_rank)
        return e, v
    r = ranks_or_rank
    buf = torch.cat([r.e_tot.reshape(-1), r.vir.reshape(-1)]).double()
    dist.all_reduce(buf)
    return buf[:1], buf[1:].reshape(1, 9)

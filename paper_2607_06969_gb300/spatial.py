"""Slab decomposition of one periodic configuration along x, evaluated from
a whole-system state that the caller holds: the building blocks of the
multi-GPU MD in halo.py (its local system and list types), and a way to
evaluate one slab of a system that is known in full.

A slab's local system holds its owned atoms (x in the slab) and the ghost
atoms within halo = 2 (rc + skin) of the slab (nep_domain_select), gathered
into a frame whose x runs over [0, slab + 2 halo + pad), with pad > rc + skin
so that the local periodic image in x never comes within the list cutoff
(nep_domain_gather).  The owned atoms are evaluated with the energy and
virial summed over them only (nep_energy_forces_virial_owned) and their
force rows scattered back (nep_domain_scatter).

With halo = 2 (rc + skin), each owned atom's neighbours (the first ghost
layer) see their whole neighbourhood (the second layer), so the owned atoms'
forces, energies and per-atom virials are those of the whole-system
evaluation, up to the order of FP32 sums.  The slab plus two halos must fit
in the box: slab + 2 halo <= L_x.  MD over several GPUs keeps no
whole-system state: halo.py moves only ghost positions between neighbouring
ranks.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as nb


def plan_slabs(Lx: float, world: int, rc: float, skin: float) -> tuple[list[tuple[float, float]], float]:
    """Equal slabs [lo, hi) of [0, Lx) per rank and the halo 2 (rc + skin);
    raises if a slab and its two halos do not fit in the box.  One rank gets
    the whole box, which needs no decomposition: nep_domain_select rejects
    it (an atom would be its own ghost), so a single GPU runs the
    whole-system calls instead."""
    if world < 1:
        raise ValueError("world must be >= 1")
    halo = 2.0 * (rc + skin)
    w = Lx / world
    if world > 1 and w + 2.0 * halo > Lx:
        raise ValueError(f"{world} slabs of {w:.2f} A with halos of {halo:.2f} A do not fit in {Lx:.2f} A")
    edges = [Lx * r / world for r in range(world + 1)]
    return [(float(edges[r]), float(edges[r + 1])) for r in range(world)], halo


class LocalSystem:
    """A device-resident single-configuration system of up to `cap` atoms
    (the local system of one slab).  Its arrays are allocated once; resize(n)
    re-points the nep_system at the first n atoms ([3][n] is the contiguous
    head of the [3 cap] buffer)."""

    def __init__(self, cap: int, box, device="cuda"):
        import torch
        self.cap = max(cap, 1)
        self.pos_buf = torch.zeros(3 * self.cap, dtype=torch.float32, device=device)
        self.type = torch.zeros(self.cap, dtype=torch.int32, device=device)
        self.box_host = np.ascontiguousarray(np.asarray(box, np.float32).reshape(1, 3))
        self.box = torch.from_numpy(self.box_host).to(device)
        self.atom_off_host = np.zeros(2, np.int32)
        self.atom_off = torch.zeros(2, dtype=torch.int32, device=device)
        self.resize(0)

    def resize(self, n: int) -> None:
        import torch
        if n > self.cap:
            raise ValueError(f"{n} atoms exceed the local capacity {self.cap}")
        self.n_atoms, self.n_cfg = n, 1
        self.pos = self.pos_buf[:3 * max(n, 1)].view(3, max(n, 1))
        self.atom_off_host[1] = n
        self.atom_off.copy_(torch.from_numpy(self.atom_off_host))
        self.c = nb.System(n, 1, self.pos.data_ptr(), self.type.data_ptr(), self.atom_off.data_ptr(),
                           self.box.data_ptr(), self.atom_off_host.ctypes.data, self.box_host.ctypes.data)


class LocalList:
    """A minimum-image Verlet list for up to `cap_atoms` atoms, allocated
    once; resize(n) re-points the nep_nlist at n atoms (slot-major arrays
    [cap][n] are the contiguous head of each buffer)."""

    def __init__(self, cap_atoms: int, cap: int, cap_ang: int, device="cuda"):
        import torch
        self.cap_atoms, self.cap, self.cap_ang = max(cap_atoms, 1), cap, cap_ang
        z = dict(dtype=torch.int32, device=device)
        self.cnt_buf = torch.zeros(self.cap_atoms, **z)
        self.cnt_ang_buf = torch.zeros(self.cap_atoms, **z)
        self.nbr_buf = torch.zeros(cap * self.cap_atoms, **z)
        self.rev_buf = torch.zeros(cap_ang * self.cap_atoms, **z)
        self.status = torch.zeros(4, **z)
        self.resize(0)

    def resize(self, n: int) -> None:
        if n > self.cap_atoms:
            raise ValueError(f"{n} atoms exceed the list capacity {self.cap_atoms}")
        self.n_atoms = n
        self.c = nb.NList(self.cap, self.cap_ang, self.cnt_buf.data_ptr(), self.cnt_ang_buf.data_ptr(),
                          self.nbr_buf.data_ptr(), 0, self.rev_buf.data_ptr(), self.status.data_ptr(), 0.0, 0)


class SlabDomain:
    """One rank's slab of a single-configuration system `gsys`
    (binding.DeviceSystem with n_cfg == 1)."""

    def __init__(self, model: nb.Model, gsys: nb.DeviceSystem, lo: float, hi: float, halo: float, skin: float,
                 cap: int, cap_ang: int, local_cap: int | None = None):
        import torch
        if gsys.n_cfg != 1:
            raise ValueError("the spatial decomposition takes one configuration")
        self.model, self.g = model, gsys
        self.lo, self.hi, self.halo, self.skin = lo, hi, halo, skin
        self.cap, self.cap_ang = cap, cap_ang
        L = gsys.box_host[0]
        h = model.h
        self.origin = lo - halo
        pad = h.rc_rad + skin + 1.0
        self.box_local = np.array([hi - lo + 2.0 * halo + pad, L[1], L[2]], np.float32)
        N = gsys.n_atoms
        if local_cap is None:
            local_cap = int(1.2 * N * min(1.0, (hi - lo + 2.0 * halo) / L[0])) + 64
        self.local_cap = local_cap
        dev = gsys.pos.device
        self.idx = torch.zeros(local_cap, dtype=torch.int32, device=dev)
        self.img = torch.zeros(local_cap, dtype=torch.int32, device=dev)
        self.counts = torch.zeros(2, dtype=torch.int32, device=dev)
        self.sel_bytes = int(nb.lib().nep_domain_workspace_bytes(N))
        self.sel_work = torch.empty(self.sel_bytes + 256, dtype=torch.uint8, device=dev)
        self.n_owned = self.n_local = 0
        self.loc = None

    def _select(self, stream=None) -> tuple[int, int]:
        w = ctypes.c_void_p(self.sel_work.data_ptr() + (-self.sel_work.data_ptr()) % 256)
        nb.check(nb.lib().nep_domain_select(
            nb._ptr(self.g.pos), self.g.n_atoms, self.g.box_host.ctypes.data_as(ctypes.c_void_p),
            ctypes.c_float(self.lo), ctypes.c_float(self.hi), ctypes.c_float(self.halo), nb._ptr(self.idx),
            nb._ptr(self.img), self.local_cap, nb._ptr(self.counts), w, self.sel_bytes, nb._stream(stream)),
            "nep_domain_select")
        c = self.counts.cpu().numpy()
        return int(c[0]), int(c[1])

    def rebuild(self, stream=None) -> None:
        """Select the owned atoms and the ghosts (positions wrapped into the
        box), gather them and build the local list.  The local arrays are
        allocated at the first call and grown only when the selection
        outgrows them."""
        import torch
        n_owned, n_local = self._select(stream)
        if n_local > self.local_cap:
            self.local_cap = int(1.2 * n_local) + 64
            dev = self.g.pos.device
            self.idx = torch.zeros(self.local_cap, dtype=torch.int32, device=dev)
            self.img = torch.zeros(self.local_cap, dtype=torch.int32, device=dev)
            n_owned, n_local = self._select(stream)
        if self.loc is None or n_local > self.loc.cap:
            dev = self.g.pos.device
            self.loc = LocalSystem(self.local_cap, self.box_local, dev)
            self.nl = LocalList(self.local_cap, self.cap, self.cap_ang, dev)
            self.ws = nb.Workspace(self.model, self.local_cap, 1, self.cap, self.cap_ang)
            self.force_buf = torch.zeros(3 * self.local_cap, dtype=torch.float32, device=dev)
            self.e_tot = torch.zeros(1, dtype=torch.float64, device=dev)
            self.vir = torch.zeros(1, 9, dtype=torch.float64, device=dev)
        self.n_owned, self.n_local = n_owned, n_local
        self.loc.resize(n_local)
        self.nl.resize(n_local)
        self.force = self.force_buf[:3 * max(n_local, 1)].view(3, max(n_local, 1))
        self.gather(stream)
        nb.neighbors(self.model, self.loc, self.nl, self.skin, self.ws, stream)

    def gather(self, stream=None) -> None:
        nb.check(nb.lib().nep_domain_gather(
            nb._ptr(self.g.pos), nb._ptr(self.g.type), self.g.n_atoms, nb._ptr(self.idx), nb._ptr(self.img),
            self.n_local, self.g.box_host.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(self.origin),
            nb._ptr(self.loc.pos), nb._ptr(self.loc.type), nb._stream(stream)), "nep_domain_gather")

    def evaluate(self, force_global, stream=None, e_atom_global=None):
        """Forces of the owned atoms into force_global [3][N] (other entries
        untouched), and the owned energy [1] and virial [1, 9] sums.  With
        e_atom_global [N], the owned atoms' energies E_i go there too."""
        import torch
        self.gather(stream)
        e_loc = None
        if e_atom_global is not None:
            nb._dev(e_atom_global, torch.float32, self.g.n_atoms, "e_atom_global", "SlabDomain.evaluate")
            if getattr(self, "e_atom", None) is None or self.e_atom.numel() < self.local_cap:
                self.e_atom = torch.zeros(self.local_cap, dtype=torch.float32, device=self.g.pos.device)
            e_loc = self.e_atom
        nb.check(nb.lib().nep_energy_forces_virial_owned(
            self.model.handle, ctypes.byref(self.loc.c), ctypes.byref(self.nl.c), self.n_owned, nb._ptr(e_loc),
            nb._ptr(self.force), nb._ptr(self.e_tot), nb._ptr(self.vir), self.ws.ptr, self.ws.bytes,
            nb._stream(stream)), "nep_energy_forces_virial_owned")
        nb.check(nb.lib().nep_domain_scatter(
            nb._ptr(self.force), self.n_local, 3, nb._ptr(self.idx), self.n_owned, nb._ptr(force_global),
            self.g.n_atoms, nb._stream(stream)), "nep_domain_scatter")
        if e_loc is not None:
            nb.check(nb.lib().nep_domain_scatter(
                nb._ptr(e_loc), self.n_local, 1, nb._ptr(self.idx), self.n_owned, nb._ptr(e_atom_global),
                self.g.n_atoms, nb._stream(stream)), "nep_domain_scatter")
        return self.e_tot, self.vir

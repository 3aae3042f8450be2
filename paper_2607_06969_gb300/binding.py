"""Python binding of libnep's C ABI (include/nep.h).

Argument marshalling only: every step of the path runs in libnep's CUDA
kernels.  PyTorch provides device memory and streams.  If libnep.so is
missing, lib() raises; nothing falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("NEP_LIB_PATH") or os.path.join(HERE, "libnep.so")

NEP_OK, NEP_ERR_ARG, NEP_ERR_CUDA, NEP_ERR_NOMEM, NEP_ERR_CAPACITY, NEP_ERR_TIMEOUT, \
    NEP_ERR_STATE, NEP_ERR_UNSUPPORTED, NEP_ERR_INPUT = range(9)

# names of every entry point declared in include/nep.h
ENTRY_POINTS = (
    "nep_num_params", "nep_create", "nep_destroy", "nep_supported", "nep_set_params", "nep_get_params",
    "nep_workspace_bytes", "nep_train_workspace_bytes", "nep_neighbors", "nep_energy_forces_virial",
    "nep_energy_forces_virial_noalloc", "nep_workspace_bytes_fp64", "nep_energy_forces_virial_fp64",
    "nep_train_workspace_bytes_fp64", "nep_param_grad_fp64", "nep_param_grad_adjoint_fp64",
    "nep_energy_forces_virial_owned", "nep_domain_workspace_bytes", "nep_domain_select", "nep_domain_gather",
    "nep_domain_scatter", "nep_domain_band", "nep_domain_take", "nep_domain_place", "nep_md_kick", "nep_md_wrap",
    "nep_param_grad",
    "nep_param_grad_adjoint", "nep_adam_step", "nep_md_step", "nep_autotune", "nep_set_variant", "nep_set_launch",
    "nep_set_timing_events", "nep_fp32_peak", "nep_selftest_wait_timeout",
    "nep_check",
    "nep_last_error", "nep_version",
)


class Hparams(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int), ("n_rad", ctypes.c_int), ("n_ang", ctypes.c_int),
                ("k_rad", ctypes.c_int), ("k_ang", ctypes.c_int), ("l_max", ctypes.c_int),
                ("has_4body", ctypes.c_int), ("n_hidden", ctypes.c_int),
                ("rc_rad", ctypes.c_float), ("rc_ang", ctypes.c_float),
                ("precision", ctypes.c_int)]


class System(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("n_cfg", ctypes.c_int),
                ("pos", ctypes.c_void_p), ("type", ctypes.c_void_p),
                ("atom_off", ctypes.c_void_p), ("box", ctypes.c_void_p),
                ("atom_off_host", ctypes.c_void_p), ("box_host", ctypes.c_void_p)]


class NList(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_int), ("cap_ang", ctypes.c_int),
                ("cnt", ctypes.c_void_p), ("cnt_ang", ctypes.c_void_p),
                ("nbr", ctypes.c_void_p), ("shift", ctypes.c_void_p),
                ("rev", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("skin", ctypes.c_float), ("min_image", ctypes.c_int)]


_LIB = None


def lib() -> ctypes.CDLL:
    """Load libnep.so (built in-tree by paper_2607_06969_gb300.build)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, f, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
    P = ctypes.POINTER
    L.nep_num_params.argtypes = [P(Hparams)]
    L.nep_num_params.restype = sz
    L.nep_supported.argtypes = [P(Hparams)]
    L.nep_supported.restype = i
    L.nep_create.argtypes = [P(Hparams), vp, sz, P(vp)]
    L.nep_destroy.argtypes = [vp]
    L.nep_set_params.argtypes = [vp, vp, vp]
    L.nep_get_params.argtypes = [vp, vp, vp]
    L.nep_adam_step.argtypes = [vp, vp, vp, vp, i, f, f, f, f, vp]
    L.nep_workspace_bytes.argtypes = [vp, i, i, i, i]
    L.nep_workspace_bytes.restype = sz
    L.nep_train_workspace_bytes.argtypes = [vp, i, i, i, i]
    L.nep_train_workspace_bytes.restype = sz
    L.nep_neighbors.argtypes = [vp, P(System), f, P(NList), vp, sz, vp]
    L.nep_energy_forces_virial.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, vp, sz, vp]
    L.nep_energy_forces_virial_noalloc.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, vp]
    L.nep_workspace_bytes_fp64.argtypes = [vp, i, i]
    L.nep_workspace_bytes_fp64.restype = sz
    L.nep_energy_forces_virial_fp64.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, vp, vp, sz, vp]
    L.nep_energy_forces_virial_owned.argtypes = [vp, P(System), P(NList), i, vp, vp, vp, vp, vp, sz, vp]
    L.nep_md_kick.argtypes = [vp, P(System), vp, vp, vp, f, f, vp]
    L.nep_md_wrap.argtypes = [vp, P(System), vp]
    L.nep_domain_workspace_bytes.argtypes = [i]
    L.nep_domain_workspace_bytes.restype = sz
    L.nep_domain_select.argtypes = [vp, i, vp, f, f, f, vp, vp, i, vp, vp, sz, vp]
    L.nep_domain_gather.argtypes = [vp, vp, i, vp, vp, i, vp, f, vp, vp, vp]
    L.nep_domain_scatter.argtypes = [vp, i, i, vp, i, vp, i, vp]
    L.nep_domain_band.argtypes = [vp, i, f, f, vp, i, vp, vp, sz, vp]
    L.nep_domain_take.argtypes = [vp, i, i, vp, i, vp, vp]
    L.nep_domain_place.argtypes = [vp, i, i, f, f, f, vp, i, i, vp]
    L.nep_train_workspace_bytes_fp64.argtypes = [vp, i, i]
    L.nep_train_workspace_bytes_fp64.restype = sz
    L.nep_param_grad_fp64.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, vp, i, vp, vp, vp, sz, vp]
    L.nep_param_grad_adjoint_fp64.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, vp, vp, sz, vp]
    L.nep_param_grad.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, i, vp, vp, vp, sz, vp]
    L.nep_param_grad_adjoint.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, vp, sz, vp]
    L.nep_md_step.argtypes = [vp, P(System), P(NList), vp, vp, vp, vp, vp, f, f, i, vp, sz, vp]
    L.nep_check.argtypes = [P(NList), vp]
    L.nep_set_timing_events.argtypes = [vp, P(vp), i]
    L.nep_autotune.argtypes = [vp, P(System), P(NList), vp, sz, vp, i, P(ctypes.c_int)]
    L.nep_autotune.restype = i
    L.nep_set_variant.argtypes = [vp, i, i]
    L.nep_set_launch.argtypes = [vp, i, i, i, i]
    L.nep_set_launch.restype = i
    L.nep_fp32_peak.argtypes = [vp, P(ctypes.c_double)]
    L.nep_fp32_peak.restype = i
    L.nep_selftest_wait_timeout.argtypes = [vp]
    L.nep_selftest_wait_timeout.restype = i
    L.nep_set_variant.restype = i
    L.nep_last_error.restype = ctypes.c_char_p
    L.nep_version.restype = ctypes.c_char_p
    for name in ("nep_create", "nep_destroy", "nep_set_params", "nep_get_params", "nep_adam_step",
                 "nep_neighbors",
                 "nep_energy_forces_virial", "nep_energy_forces_virial_noalloc",
                 "nep_energy_forces_virial_fp64", "nep_param_grad_fp64", "nep_param_grad_adjoint_fp64",
                 "nep_energy_forces_virial_owned", "nep_domain_select", "nep_domain_gather",
                 "nep_domain_scatter", "nep_domain_band", "nep_domain_take", "nep_domain_place",
                 "nep_md_kick", "nep_md_wrap",
                 "nep_param_grad", "nep_param_grad_adjoint",
                 "nep_md_step", "nep_check", "nep_set_timing_events"):
        getattr(L, name).restype = i
    _LIB = L
    return L


class NepError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != NEP_OK:
        raise NepError(status, where, lib().nep_last_error().decode())


def hparams_of(h, precision: int = 0) -> Hparams:
    return Hparams(h.n_types, h.n_rad, h.n_ang, h.k_rad, h.k_ang, h.l_max, h.has_4body,
                   h.n_hidden, float(h.rc_rad), float(h.rc_ang), precision)


def num_params(h) -> int:
    hp = hparams_of(h)
    return int(lib().nep_num_params(ctypes.byref(hp)))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _dev(t, dtype, numel: int, name: str, where: str, optional: bool = False):
    """A device argument of a library call: a contiguous CUDA tensor of
    `dtype` with at least `numel` elements (the count the call reads or
    writes), or None where the call accepts NULL.  Raises ValueError
    otherwise, so that a wrong tensor never reaches the device."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{where}: {name} is required")
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() >= numel):
        raise ValueError(f"{where}: {name} must be a contiguous CUDA {dtype} tensor of at least {numel} "
                         f"elements (got {t.dtype}, shape {tuple(t.shape)}, "
                         f"{'cuda' if t.is_cuda else 'cpu'}, {'' if t.is_contiguous() else 'not '}contiguous)")
    return t


def _outputs(dsys, out, dtype, where: str):
    """(e_atom [N] or None, force [3,N], e_tot [B], virial [B,9]) checked."""
    import torch
    e_atom, force, e_tot, vir = out
    _dev(e_atom, dtype, dsys.n_atoms, "e_atom", where, optional=True)
    _dev(force, dtype, 3 * dsys.n_atoms, "force", where)
    _dev(e_tot, torch.float64, dsys.n_cfg, "e_tot", where)
    _dev(vir, torch.float64, 9 * dsys.n_cfg, "virial", where)
    return out


def _labels(dsys, e_lbl, f_lbl, v_lbl, f_dtype, where: str) -> None:
    """Labels E [B] f64, F [3,N] (f_dtype), V [B,9] f64."""
    import torch
    _dev(e_lbl, torch.float64, dsys.n_cfg, "e_lbl", where)
    _dev(f_lbl, f_dtype, 3 * dsys.n_atoms, "f_lbl", where)
    _dev(v_lbl, torch.float64, 9 * dsys.n_cfg, "v_lbl", where)


def _adjoints(dsys, a_e, lam, mu, lam_dtype, where: str) -> None:
    """Adjoints a_e [B] f64, lam [3,N] (lam_dtype), mu [B,9] f64."""
    import torch
    _dev(a_e, torch.float64, dsys.n_cfg, "a_e", where)
    _dev(lam, lam_dtype, 3 * dsys.n_atoms, "lam", where)
    _dev(mu, torch.float64, 9 * dsys.n_cfg, "mu", where)


def _weights(w, where: str) -> np.ndarray:
    """The loss weights (wE, wF, wV) as a host float array."""
    wh = np.ascontiguousarray(np.asarray(w, np.float32).reshape(-1))
    if wh.size != 3:
        raise ValueError(f"{where}: w must hold the three weights (wE, wF, wV)")
    return wh


def _same_atoms(dsys, nl, where: str) -> None:
    """The list's per-atom arrays must be sized for the system's atoms (the
    library indexes them by the system's atom count)."""
    n = getattr(nl, "n_atoms", None)
    if nl is not None and n != dsys.n_atoms:
        raise ValueError(f"{where}: the neighbour list holds {n} atoms, the system {dsys.n_atoms}")


def _stream(stream=None) -> ctypes.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Model:
    """A NEP model on the current CUDA device (nep_create / nep_destroy)."""

    def __init__(self, h, params, precision: int = 0):
        self.h = h
        self.hp = hparams_of(h, precision)
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        self.n_params = p.size
        handle = ctypes.c_void_p()
        check(lib().nep_create(ctypes.byref(self.hp), p.ctypes.data_as(ctypes.c_void_p),
                               p.size, ctypes.byref(handle)), "nep_create")
        self.handle = handle

    def set_params(self, params_dev, stream=None):
        import torch
        _dev(params_dev, torch.float32, self.n_params, "params", "nep_set_params")
        check(lib().nep_set_params(self.handle, _ptr(params_dev), _stream(stream)), "nep_set_params")

    def get_params(self, out=None, stream=None):
        """nep_get_params: the current parameters as a device tensor [P] f32."""
        import torch
        if out is None:
            out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _dev(out, torch.float32, self.n_params, "out", "nep_get_params")
        check(lib().nep_get_params(self.handle, _ptr(out), _stream(stream)), "nep_get_params")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().nep_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceSystem:
    """A batch of periodic configurations resident on the GPU (nep_system)."""

    def __init__(self, pos, types, box, atom_off, device="cuda"):
        """pos [N,3], types [N], box [B,3] (orthorhombic edges), atom_off [B+1]
        on the host; the shapes are checked here, the values by the library."""
        import torch
        pos = np.asarray(pos, np.float32)
        types = np.asarray(types, np.int32)
        box = np.asarray(box, np.float32)
        atom_off = np.asarray(atom_off, np.int32)
        if pos.ndim != 2 or pos.shape[1] != 3:
            raise ValueError(f"pos must be [N, 3], got {pos.shape}")
        if types.shape != (pos.shape[0],):
            raise ValueError(f"types must be [N] = [{pos.shape[0]}], got {types.shape}")
        if box.ndim != 2 or box.shape[1] != 3:
            raise ValueError(f"box must be [B, 3], got {box.shape}")
        if atom_off.shape != (box.shape[0] + 1,):
            raise ValueError(f"atom_off must be [B + 1] = [{box.shape[0] + 1}], got {atom_off.shape}")
        self.n_atoms = int(pos.shape[0])
        self.n_cfg = int(box.shape[0])
        self.pos = torch.from_numpy(np.ascontiguousarray(pos.T)).to(device)        # [3][N]
        self.type = torch.from_numpy(np.ascontiguousarray(types)).to(device)
        self.atom_off_host = np.ascontiguousarray(atom_off)
        self.box_host = np.ascontiguousarray(box)
        self.atom_off = torch.from_numpy(self.atom_off_host).to(device)
        self.box = torch.from_numpy(self.box_host).to(device)
        self.refresh()

    @classmethod
    def from_inputs(cls, s, device="cuda"):
        return cls(s.pos32(), s.types, s.box, s.atom_off, device)

    def refresh(self):
        self.c = System(self.n_atoms, self.n_cfg, self.pos.data_ptr(), self.type.data_ptr(),
                        self.atom_off.data_ptr(), self.box.data_ptr(),
                        self.atom_off_host.ctypes.data, self.box_host.ctypes.data)
        return self.c


class NeighborList:
    """Caller-owned Verlet list (nep_nlist) with capacities cap >= cap_ang."""

    def __init__(self, n_atoms: int, cap: int, cap_ang: int, shifts: bool = True, device="cuda"):
        import torch
        self.n_atoms, self.cap, self.cap_ang = n_atoms, cap, cap_ang
        z = dict(dtype=torch.int32, device=device)
        self.cnt = torch.zeros(n_atoms, **z)
        self.cnt_ang = torch.zeros(n_atoms, **z)
        self.nbr = torch.zeros(cap * n_atoms, **z)
        self.shift = torch.zeros(cap * n_atoms, **z) if shifts else None
        self.rev = torch.zeros(cap_ang * n_atoms, **z)
        self.status = torch.zeros(4, **z)
        self.c = NList(cap, cap_ang, self.cnt.data_ptr(), self.cnt_ang.data_ptr(),
                       self.nbr.data_ptr(), 0 if self.shift is None else self.shift.data_ptr(),
                       self.rev.data_ptr(), self.status.data_ptr(), 0.0, 0)

    def to_pairs(self, box=None):
        """(i, j, s) arrays of the radial list, and the angular prefix mask."""
        N = self.n_atoms
        cnt = self.cnt.cpu().numpy()
        cnta = self.cnt_ang.cpu().numpy()
        nbr = self.nbr.cpu().numpy().reshape(self.cap, N)
        slot = np.arange(self.cap)[:, None]
        mask = slot < cnt[None, :]
        ii = np.broadcast_to(np.arange(N)[None, :], (self.cap, N))[mask]
        jj = nbr[mask]
        ang = (slot < cnta[None, :])[mask]
        if self.shift is not None and not self.c.min_image:
            sh = self.shift.cpu().numpy().reshape(self.cap, N)[mask]
            s = np.stack([((sh >> (8 * k)) & 0xff).astype(np.int8).astype(np.int64) for k in range(3)], 1)
        else:
            s = None
        return ii.astype(np.int64), jj.astype(np.int64), s, ang


class Workspace:
    """Device scratch for the hot calls (nep_workspace_bytes, or
    nep_train_workspace_bytes with train=True)."""

    def __init__(self, model: Model, n_atoms: int, n_cfg: int, cap: int, cap_ang: int, device="cuda",
                 train: bool = False):
        import torch
        fn = lib().nep_train_workspace_bytes if train else lib().nep_workspace_bytes
        self.bytes = int(fn(model.handle, n_atoms, n_cfg, cap, cap_ang))
        if self.bytes == 0:
            raise NepError(NEP_ERR_ARG, "nep_workspace_bytes", "invalid sizes")
        self.buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = ctypes.c_void_p(self.buf.data_ptr() + off)


def neighbors(model: Model, dsys: DeviceSystem, nl: NeighborList, skin: float, ws: Workspace,
              stream=None) -> None:
    _same_atoms(dsys, nl, "nep_neighbors")
    check(lib().nep_neighbors(model.handle, ctypes.byref(dsys.c), float(skin), ctypes.byref(nl.c),
                              ws.ptr, ws.bytes, _stream(stream)), "nep_neighbors")


def energy_forces_virial(model: Model, dsys: DeviceSystem, nl: NeighborList, ws: Workspace,
                         out=None, stream=None):
    """Returns (e_atom [N] f32, force [3,N] f32, e_tot [B] f64, virial [B,9] f64)."""
    _same_atoms(dsys, nl, "nep_energy_forces_virial")
    import torch
    dev = dsys.pos.device
    if out is None:
        out = (torch.empty(dsys.n_atoms, dtype=torch.float32, device=dev),
               torch.empty(3, dsys.n_atoms, dtype=torch.float32, device=dev),
               torch.empty(dsys.n_cfg, dtype=torch.float64, device=dev),
               torch.empty(dsys.n_cfg, 9, dtype=torch.float64, device=dev))
    e_atom, force, e_tot, vir = _outputs(dsys, out, torch.float32, "nep_energy_forces_virial")
    check(lib().nep_energy_forces_virial(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c),
                                         _ptr(e_atom), _ptr(force), _ptr(e_tot), _ptr(vir),
                                         ws.ptr, ws.bytes, _stream(stream)),
          "nep_energy_forces_virial")
    return out


class Workspace64:
    """Device scratch of the FP64 calls (nep_workspace_bytes_fp64, or
    nep_train_workspace_bytes_fp64 with train=True)."""

    def __init__(self, model: Model, n_atoms: int, n_cfg: int, device="cuda", train: bool = False):
        import torch
        fn = lib().nep_train_workspace_bytes_fp64 if train else lib().nep_workspace_bytes_fp64
        self.bytes = int(fn(model.handle, n_atoms, n_cfg))
        if self.bytes == 0:
            raise NepError(NEP_ERR_ARG, "nep_workspace_bytes_fp64", "invalid sizes")
        self.buf = torch.empty(self.bytes + 256, dtype=torch.uint8, device=device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = ctypes.c_void_p(self.buf.data_ptr() + off)


def energy_forces_virial_fp64(model: Model, dsys: DeviceSystem, nl: NeighborList, ws: Workspace64,
                              params=None, out=None, stream=None):
    """nep_energy_forces_virial_fp64: (e_atom [N], force [3,N], e_tot [B],
    virial [B,9]), all f64.  params: optional device tensor [P] f64 (default:
    the model's FP32 parameters promoted)."""
    _same_atoms(dsys, nl, "nep_energy_forces_virial_fp64")
    import torch
    dev = dsys.pos.device
    _dev(params, torch.float64, model.n_params, "params", "nep_energy_forces_virial_fp64", optional=True)
    if out is None:
        out = (torch.empty(dsys.n_atoms, dtype=torch.float64, device=dev),
               torch.empty(3, dsys.n_atoms, dtype=torch.float64, device=dev),
               torch.empty(dsys.n_cfg, dtype=torch.float64, device=dev),
               torch.empty(dsys.n_cfg, 9, dtype=torch.float64, device=dev))
    e_atom, force, e_tot, vir = _outputs(dsys, out, torch.float64, "nep_energy_forces_virial_fp64")
    check(lib().nep_energy_forces_virial_fp64(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c),
                                              _ptr(params), _ptr(e_atom), _ptr(force), _ptr(e_tot),
                                              _ptr(vir), ws.ptr, ws.bytes, _stream(stream)),
          "nep_energy_forces_virial_fp64")
    return out


def param_grad_fp64(model: Model, dsys: DeviceSystem, nl: NeighborList, ws: Workspace64, e_lbl, f_lbl,
                    v_lbl, w=(1.0, 1.0, 0.1), loss_mode: int = 0, params=None, grad=None, loss=None,
                    stream=None):
    """nep_param_grad_fp64: (grad [P] f64, loss [1] f64); labels e_lbl [B],
    f_lbl [3,N], v_lbl [B,9] f64 on the device; ws a training Workspace64."""
    _same_atoms(dsys, nl, "nep_param_grad_fp64")
    import torch
    dev = dsys.pos.device
    where, f64 = "nep_param_grad_fp64", torch.float64
    _labels(dsys, e_lbl, f_lbl, v_lbl, f64, where)
    _dev(params, f64, model.n_params, "params", where, optional=True)
    if grad is None:
        grad = torch.empty(model.n_params, dtype=f64, device=dev)
    if loss is None:
        loss = torch.empty(1, dtype=f64, device=dev)
    _dev(grad, f64, model.n_params, "grad", where)
    _dev(loss, f64, 1, "loss", where)
    wh = _weights(w, where)
    check(lib().nep_param_grad_fp64(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c), _ptr(params),
                                    _ptr(e_lbl), _ptr(f_lbl), _ptr(v_lbl), wh.ctypes.data_as(ctypes.c_void_p),
                                    int(loss_mode), _ptr(grad), _ptr(loss), ws.ptr, ws.bytes, _stream(stream)),
          "nep_param_grad_fp64")
    return grad, loss


def param_grad_adjoint_fp64(model: Model, dsys: DeviceSystem, nl: NeighborList, ws: Workspace64, a_e, lam,
                            mu, params=None, grad=None, stream=None):
    """nep_param_grad_adjoint_fp64: grad [P] f64 of sum a_e E + lam . F +
    mu : V (a_e [B], lam [3,N], mu [B,9] f64 on the device)."""
    _same_atoms(dsys, nl, "nep_param_grad_adjoint_fp64")
    import torch
    dev = dsys.pos.device
    where, f64 = "nep_param_grad_adjoint_fp64", torch.float64
    _adjoints(dsys, a_e, lam, mu, f64, where)
    _dev(params, f64, model.n_params, "params", where, optional=True)
    if grad is None:
        grad = torch.empty(model.n_params, dtype=f64, device=dev)
    _dev(grad, f64, model.n_params, "grad", where)
    check(lib().nep_param_grad_adjoint_fp64(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c),
                                            _ptr(params), _ptr(a_e), _ptr(lam), _ptr(mu), _ptr(grad), ws.ptr,
                                            ws.bytes, _stream(stream)),
          "nep_param_grad_adjoint_fp64")
    return grad


def param_grad(model: Model, dsys: DeviceSystem, nl: NeighborList, ws: Workspace, e_lbl, f_lbl,
               v_lbl, w=(1.0, 1.0, 0.1), loss_mode: int = 0, grad=None, loss=None, stream=None):
    """nep_param_grad: loss (Eqs. 18-21) and its gradient over all parameters.
    e_lbl [B] f64, f_lbl [3,N] f32, v_lbl [B,9] f64 on the device; ws must be a
    training workspace.  Returns (grad [P] f32, loss [1] f64)."""
    _same_atoms(dsys, nl, "nep_param_grad")
    import torch
    dev = dsys.pos.device
    where = "nep_param_grad"
    _labels(dsys, e_lbl, f_lbl, v_lbl, torch.float32, where)
    if grad is None:
        grad = torch.empty(model.n_params, dtype=torch.float32, device=dev)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=dev)
    _dev(grad, torch.float32, model.n_params, "grad", where)
    _dev(loss, torch.float64, 1, "loss", where)
    wh = _weights(w, where)
    check(lib().nep_param_grad(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c), _ptr(e_lbl),
                               _ptr(f_lbl), _ptr(v_lbl), wh.ctypes.data_as(ctypes.c_void_p),
                               int(loss_mode), _ptr(grad), _ptr(loss), ws.ptr, ws.bytes, _stream(stream)),
          "nep_param_grad")
    return grad, loss


def param_grad_adjoint(model: Model, dsys: DeviceSystem, nl: NeighborList, ws: Workspace, a_e, lam, mu,
                       grad=None, stream=None):
    """nep_param_grad_adjoint: d/dtheta of sum a_e E + lam . F + mu : V.
    a_e [B] f64, lam [3,N] f32, mu [B,9] f64.  Returns grad [P] f32."""
    _same_atoms(dsys, nl, "nep_param_grad_adjoint")
    import torch
    where = "nep_param_grad_adjoint"
    _adjoints(dsys, a_e, lam, mu, torch.float32, where)
    if grad is None:
        grad = torch.empty(model.n_params, dtype=torch.float32, device=dsys.pos.device)
    _dev(grad, torch.float32, model.n_params, "grad", where)
    check(lib().nep_param_grad_adjoint(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c),
                                       _ptr(a_e), _ptr(lam), _ptr(mu), _ptr(grad), ws.ptr, ws.bytes,
                                       _stream(stream)), "nep_param_grad_adjoint")
    return grad


def adam_step(model: Model, grad, m1, m2, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, stream=None) -> None:
    """nep_adam_step: one Adam update of the model's parameters in place.
    grad, m1, m2: device tensors [P] f32 (m1, m2 zero before t = 1)."""
    import torch
    for name, x in (("grad", grad), ("m1", m1), ("m2", m2)):
        _dev(x, torch.float32, model.n_params, name, "nep_adam_step")
    check(lib().nep_adam_step(model.handle, _ptr(grad), _ptr(m1), _ptr(m2), int(t), float(lr), float(beta1),
                              float(beta2), float(eps), _stream(stream)), "nep_adam_step")


NOALLOC_SCRATCH_BYTES = 32 << 20


def energy_forces_virial_noalloc(model: Model, dsys: DeviceSystem, nl: NeighborList, out=None,
                                 stream=None):
    """nep_energy_forces_virial_noalloc: the same outputs as
    energy_forces_virial, with scratch taken from the library's static
    device array instead of a caller workspace (for callers that cannot
    allocate device memory).  Returns (e_atom, force [3,N], e_tot, virial)."""
    _same_atoms(dsys, nl, "nep_energy_forces_virial_noalloc")
    import torch
    dev = dsys.pos.device
    if out is None:
        out = (torch.empty(dsys.n_atoms, dtype=torch.float32, device=dev),
               torch.empty(3, dsys.n_atoms, dtype=torch.float32, device=dev),
               torch.empty(dsys.n_cfg, dtype=torch.float64, device=dev),
               torch.empty(dsys.n_cfg, 9, dtype=torch.float64, device=dev))
    e_atom, force, e_tot, vir = _outputs(dsys, out, torch.float32, "nep_energy_forces_virial_noalloc")
    check(lib().nep_energy_forces_virial_noalloc(model.handle, ctypes.byref(dsys.c),
                                                 ctypes.byref(nl.c), _ptr(e_atom), _ptr(force),
                                                 _ptr(e_tot), _ptr(vir), _stream(stream)),
          "nep_energy_forces_virial_noalloc")
    return out


def md_step(model: Model, dsys: DeviceSystem, nl: NeighborList, vel, force, e_tot, virial,
            masses, dt: float, skin: float, rebuild: bool, ws: Workspace, stream=None) -> None:
    """nep_md_step: vel [3,N] f32 (in place), force [3,N] f32, e_tot [B] and
    virial [B,9] f64 on the device; masses: host, one per species."""
    _same_atoms(dsys, nl, "nep_md_step")
    import torch
    _outputs(dsys, (None, force, e_tot, virial), torch.float32, "nep_md_step")
    _dev(vel, torch.float32, 3 * dsys.n_atoms, "vel", "nep_md_step")
    m = np.ascontiguousarray(np.asarray(masses, np.float32))
    if m.size < model.hp.n_types:
        raise ValueError(f"nep_md_step: {m.size} masses for {model.hp.n_types} species")
    check(lib().nep_md_step(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c), _ptr(vel),
                            _ptr(force), _ptr(e_tot), _ptr(virial),
                            m.ctypes.data_as(ctypes.c_void_p), float(dt), float(skin),
                            1 if rebuild else 0, ws.ptr, ws.bytes, _stream(stream)), "nep_md_step")


def set_timing_events(model: Model, events) -> None:
    """events: four torch.cuda.Event(enable_timing=True) (before the radial
    kernel, after it, after the angular kernel(s), after the finish kernel),
    or None to clear."""
    if events is None:
        check(lib().nep_set_timing_events(model.handle, None, 0), "nep_set_timing_events")
        return
    arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in events])
    check(lib().nep_set_timing_events(model.handle, arr, 4), "nep_set_timing_events")


def autotune(model: Model, dsys: DeviceSystem, nl: NeighborList, ws: Workspace, reps: int = 3,
             stream=None):
    """nep_autotune: pick the angular kernel variant and the radial and
    finish block sizes for this system's size class; returns them as
    (variant, radial block, finish block)."""
    _same_atoms(dsys, nl, "nep_autotune")
    chosen = (ctypes.c_int * 3)()
    check(lib().nep_autotune(model.handle, ctypes.byref(dsys.c), ctypes.byref(nl.c), ws.ptr, ws.bytes,
                             _stream(stream), int(reps), chosen), "nep_autotune")
    return int(chosen[0]), int(chosen[1]), int(chosen[2])


def set_launch(model: Model, variant: int = -1, radial_block: int = 0, finish_block: int = 0,
               size_class: int = -1) -> None:
    """nep_set_launch: pin the launch choices (defaults: -1 / 0) for one size
    class or all of them."""
    check(lib().nep_set_launch(model.handle, int(size_class), int(variant), int(radial_block),
                               int(finish_block)), "nep_set_launch")


def set_variant(model: Model, variant: int, size_class: int = -1) -> None:
    """nep_set_variant: pin the angular kernel variant (-1 = default) for one
    size class or all of them."""
    check(lib().nep_set_variant(model.handle, int(size_class), int(variant)), "nep_set_variant")


def fp32_peak(stream=None) -> float:
    """nep_fp32_peak: measured FP32 FMA throughput of the device, TFLOP/s."""
    out = ctypes.c_double()
    check(lib().nep_fp32_peak(_stream(stream), ctypes.byref(out)), "nep_fp32_peak")
    return float(out.value)


def selftest_wait_timeout(stream=None) -> int:
    """nep_selftest_wait_timeout: the status of a bounded tensor-core wait
    that is made to run out (NEP_ERR_TIMEOUT when it works as designed)."""
    return int(lib().nep_selftest_wait_timeout(_stream(stream)))


def check_list(nl: NeighborList | None, stream=None) -> int:
    """nep_check: synchronise and return the status (does not raise)."""
    return int(lib().nep_check(None if nl is None else ctypes.byref(nl.c), _stream(stream)))


def last_error() -> str:
    return lib().nep_last_error().decode()

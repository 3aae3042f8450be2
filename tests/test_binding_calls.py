"""Every binding wrapper, driven on the CPU with valid stand-in tensors
through a recording stub of the library: each C call must receive the
arguments its declaration in include/nep.h names, with the types ctypes
expects (an int where the call takes an int, the tensor's address where it
takes a pointer).  The wrappers' rejections of bad tensors are tested in
test_binding_host.py; this file covers the valid calls."""
import ctypes
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from paper_2607_06969_gb300 import binding as nb
from paper_2607_06969_gb300 import inputs as I

F32, F64, I32 = torch.float32, torch.float64, torch.int32


class Dev:
    """A CUDA tensor stand-in with a distinct, recognisable address."""
    _next = 0x10000

    def __init__(self, numel, dtype=F32):
        self.is_cuda, self.dtype, self._n = True, dtype, numel
        self.shape = (numel,)
        Dev._next += 0x1000
        self.addr = Dev._next

    def numel(self):
        return self._n

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return self.addr


class StubLib:
    """Records (name, args) of every call and returns NEP_OK, or a size for
    the *_bytes queries."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if name.startswith("__"):
            raise AttributeError(name)

        def call(*args):
            self.calls.append((name, args))
            if "_bytes" in name:
                return 4096
            if name == "nep_num_params":
                return 4611
            if name in ("nep_last_error", "nep_version"):
                return b""
            if name == "nep_create":
                args[3]._obj.value = 0xABC
            if name == "nep_fp32_peak":
                args[1]._obj.value = 76.5
            if name == "nep_autotune":
                args[7][0], args[7][1], args[7][2] = 2, 64, 128
            return nb.NEP_OK
        return call

    def last(self, name):
        hits = [a for n, a in self.calls if n == name]
        assert hits, f"{name} was not called"
        return hits[-1]


STREAM = SimpleNamespace(cuda_stream=0x5151)


def addr(p):
    return p.value if isinstance(p, ctypes.c_void_p) else p


@pytest.fixture()
def stub(monkeypatch):
    s = StubLib()
    monkeypatch.setattr(nb, "lib", lambda: s)
    return s


@pytest.fixture()
def parts(stub):
    h = I.Hyper(n_types=3, n_rad=8, n_ang=6, k_rad=8, k_ang=8, l_max=4, has_4body=1, n_hidden=30,
                rc_rad=7.0, rc_ang=5.0)
    model = nb.Model(h, np.zeros(h.n_params, np.float32))
    N, B = 10, 2
    dsys = nb.DeviceSystem(np.zeros((N, 3)), np.zeros(N, np.int32), np.full((B, 3), 20.0),
                           np.array([0, 4, N]), device="cpu")
    nl = SimpleNamespace(n_atoms=N, c=nb.NList(64, 32, 0, 0, 0, 0, 0, 0, 0.0, 0))
    ws = nb.Workspace(model, N, B, 64, 32, device="cpu")
    yield SimpleNamespace(h=h, model=model, dsys=dsys, nl=nl, ws=ws, N=N, B=B, P=model.n_params)
    # the handle is the stub's: never let the real library destroy it
    model.handle = None


def test_create_passes_hparams_and_parameter_count(stub, parts):
    hp_ref, _, n, _ = stub.last("nep_create")
    hp = hp_ref._obj
    assert (hp.n_types, hp.n_rad, hp.n_ang, hp.k_rad, hp.k_ang, hp.l_max, hp.has_4body, hp.n_hidden) == \
        (3, 8, 6, 8, 8, 4, 1, 30)
    assert hp.rc_rad == 7.0 and hp.rc_ang == 5.0 and hp.precision == 0
    assert n == parts.P and parts.model.handle.value == 0xABC
    assert stub.last("nep_workspace_bytes")[1:] == (parts.N, parts.B, 64, 32)
    assert parts.ws.bytes == 4096 and parts.ws.ptr.value % 256 == 0


def test_adam_step_passes_the_integer_step_counter(stub, parts):
    g, m1, m2 = Dev(parts.P), Dev(parts.P), Dev(parts.P)
    nb.adam_step(parts.model, g, m1, m2, 7, 1e-3, 0.8, 0.99, 1e-7, stream=STREAM)
    a = stub.last("nep_adam_step")
    assert [addr(x) for x in a[1:4]] == [g.addr, m1.addr, m2.addr]
    assert type(a[4]) is int and a[4] == 7
    assert a[5:9] == pytest.approx((1e-3, 0.8, 0.99, 1e-7))
    assert all(type(x) is float for x in a[5:9])
    assert addr(a[9]) == STREAM.cuda_stream


def test_params_calls(stub, parts):
    p = Dev(parts.P)
    parts.model.set_params(p, stream=STREAM)
    assert addr(stub.last("nep_set_params")[1]) == p.addr
    out = Dev(parts.P)
    assert parts.model.get_params(out, stream=STREAM) is out
    assert addr(stub.last("nep_get_params")[1]) == out.addr


def test_evaluation_calls(stub, parts):
    N, B = parts.N, parts.B
    nb.neighbors(parts.model, parts.dsys, parts.nl, 1.0, parts.ws, stream=STREAM)
    a = stub.last("nep_neighbors")
    assert a[2] == 1.0 and type(a[2]) is float and a[5] == parts.ws.bytes
    out = (Dev(N), Dev(3 * N), Dev(B, F64), Dev(9 * B, F64))
    assert nb.energy_forces_virial(parts.model, parts.dsys, parts.nl, parts.ws, out=out, stream=STREAM) is out
    a = stub.last("nep_energy_forces_virial")
    assert [addr(x) for x in a[3:7]] == [t.addr for t in out]
    assert a[8] == parts.ws.bytes and addr(a[9]) == STREAM.cuda_stream
    out2 = (None, Dev(3 * N), Dev(B, F64), Dev(9 * B, F64))
    nb.energy_forces_virial_noalloc(parts.model, parts.dsys, parts.nl, out=out2, stream=STREAM)
    a = stub.last("nep_energy_forces_virial_noalloc")
    assert addr(a[3]) in (0, None) and [addr(x) for x in a[4:7]] == [t.addr for t in out2[1:]]


def test_training_calls(stub, parts):
    N, B, P = parts.N, parts.B, parts.P
    e, f, v = Dev(B, F64), Dev(3 * N), Dev(9 * B, F64)
    grad, loss = Dev(P), Dev(1, F64)
    nb.param_grad(parts.model, parts.dsys, parts.nl, parts.ws, e, f, v, w=(1.0, 2.0, 0.5), loss_mode=1,
                  grad=grad, loss=loss, stream=STREAM)
    a = stub.last("nep_param_grad")
    assert [addr(x) for x in a[3:6]] == [e.addr, f.addr, v.addr]
    w = np.ctypeslib.as_array(ctypes.cast(a[6], ctypes.POINTER(ctypes.c_float)), (3,))
    assert list(w) == [1.0, 2.0, 0.5]
    assert type(a[7]) is int and a[7] == 1
    assert [addr(x) for x in a[8:10]] == [grad.addr, loss.addr]
    ae, lam, mu = Dev(B, F64), Dev(3 * N), Dev(9 * B, F64)
    assert nb.param_grad_adjoint(parts.model, parts.dsys, parts.nl, parts.ws, ae, lam, mu, grad=grad,
                                 stream=STREAM) is grad
    a = stub.last("nep_param_grad_adjoint")
    assert [addr(x) for x in a[3:7]] == [ae.addr, lam.addr, mu.addr, grad.addr]


def test_fp64_calls(stub, parts):
    N, B, P = parts.N, parts.B, parts.P
    ws = nb.Workspace64(parts.model, N, B, device="cpu")
    assert stub.last("nep_workspace_bytes_fp64")[1:] == (N, B)
    out = (Dev(N, F64), Dev(3 * N, F64), Dev(B, F64), Dev(9 * B, F64))
    prm = Dev(P, F64)
    nb.energy_forces_virial_fp64(parts.model, parts.dsys, parts.nl, ws, params=prm, out=out, stream=STREAM)
    a = stub.last("nep_energy_forces_virial_fp64")
    assert addr(a[3]) == prm.addr and [addr(x) for x in a[4:8]] == [t.addr for t in out]
    e, f, v = Dev(B, F64), Dev(3 * N, F64), Dev(9 * B, F64)
    grad, loss = Dev(P, F64), Dev(1, F64)
    nb.param_grad_fp64(parts.model, parts.dsys, parts.nl, ws, e, f, v, loss_mode=0, grad=grad, loss=loss,
                       stream=STREAM)
    a = stub.last("nep_param_grad_fp64")
    assert addr(a[3]) in (0, None) and type(a[8]) is int and addr(a[9]) == grad.addr
    nb.param_grad_adjoint_fp64(parts.model, parts.dsys, parts.nl, ws, e, f, v, grad=grad, stream=STREAM)
    assert addr(stub.last("nep_param_grad_adjoint_fp64")[7]) == grad.addr


def test_md_step_passes_masses_and_rebuild_flag(stub, parts):
    N, B = parts.N, parts.B
    vel, force, et, vir = Dev(3 * N), Dev(3 * N), Dev(B, F64), Dev(9 * B, F64)
    for rebuild, flag in ((True, 1), (False, 0)):
        nb.md_step(parts.model, parts.dsys, parts.nl, vel, force, et, vir, [72.63, 121.76, 127.6], 2.0, 1.0,
                   rebuild, parts.ws, stream=STREAM)
        a = stub.last("nep_md_step")
        assert [addr(x) for x in a[3:7]] == [vel.addr, force.addr, et.addr, vir.addr]
        m = np.ctypeslib.as_array(ctypes.cast(a[7], ctypes.POINTER(ctypes.c_float)), (3,))
        assert m == pytest.approx([72.63, 121.76, 127.6])
        assert a[8] == 2.0 and a[9] == 1.0 and type(a[10]) is int and a[10] == flag


def test_tuning_and_helper_calls(stub, parts):
    assert nb.autotune(parts.model, parts.dsys, parts.nl, parts.ws, reps=4, stream=STREAM) == (2, 64, 128)
    assert stub.last("nep_autotune")[6] == 4
    nb.set_variant(parts.model, 1, 3)
    assert stub.last("nep_set_variant")[1:] == (3, 1)
    nb.set_launch(parts.model, 2, 128, 64, size_class=5)
    assert stub.last("nep_set_launch")[1:] == (5, 2, 128, 64)
    assert nb.fp32_peak(stream=STREAM) == pytest.approx(76.5)
    assert nb.selftest_wait_timeout(stream=STREAM) == nb.NEP_OK
    assert nb.check_list(parts.nl, stream=STREAM) == nb.NEP_OK
    assert nb.check_list(None, stream=STREAM) == nb.NEP_OK and stub.last("nep_check")[0] is None
    ev = [SimpleNamespace(cuda_event=0x100 + k) for k in range(4)]
    nb.set_timing_events(parts.model, ev)
    a = stub.last("nep_set_timing_events")
    assert [a[1][k] for k in range(4)] == [0x100, 0x101, 0x102, 0x103] and a[2] == 4
    nb.set_timing_events(parts.model, None)
    assert stub.last("nep_set_timing_events")[1:] == (None, 0)
    assert nb.num_params(parts.h) == 4611
    parts.model.close()
    assert addr(stub.last("nep_destroy")[0]) == 0xABC and parts.model.handle is None

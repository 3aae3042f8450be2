"""The binding's device-argument checks, on the CPU: a tensor handed to a
library call must be a contiguous CUDA tensor of the call's dtype with at
least as many elements as the call reads or writes; anything else raises
ValueError before the library is reached."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from paper_2607_06969_gb300 import binding as nb


class DeviceLike:
    """Stands in for a CUDA tensor (no GPU here): the attributes the checks read."""

    def __init__(self, numel, dtype=torch.float32, contiguous=True):
        self.is_cuda, self.dtype, self._n, self._c = True, dtype, numel, contiguous
        self.shape = (numel,)

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


def test_dev_accepts_and_rejects():
    assert nb._dev(None, torch.float32, 4, "x", "call", optional=True) is None
    t = DeviceLike(10)
    assert nb._dev(t, torch.float32, 10, "x", "call") is t
    for bad in (None, DeviceLike(9), DeviceLike(10, torch.float64), DeviceLike(10, contiguous=False),
                torch.zeros(10)):
        with pytest.raises(ValueError, match="call: x"):
            nb._dev(bad, torch.float32, 10, "x", "call")


def test_group_checks_size_by_atoms_and_configurations():
    dsys = SimpleNamespace(n_atoms=7, n_cfg=2)
    f32, f64 = torch.float32, torch.float64
    nb._outputs(dsys, (None, DeviceLike(21), DeviceLike(2, f64), DeviceLike(18, f64)), f32, "efv")
    with pytest.raises(ValueError, match="virial"):
        nb._outputs(dsys, (None, DeviceLike(21), DeviceLike(2, f64), DeviceLike(17, f64)), f32, "efv")
    with pytest.raises(ValueError, match="e_atom"):
        nb._outputs(dsys, (DeviceLike(6), DeviceLike(21), DeviceLike(2, f64), DeviceLike(18, f64)), f32, "efv")
    nb._labels(dsys, DeviceLike(2, f64), DeviceLike(21, f64), DeviceLike(18, f64), f64, "grad64")
    with pytest.raises(ValueError, match="f_lbl"):
        nb._labels(dsys, DeviceLike(2, f64), DeviceLike(21), DeviceLike(18, f64), f64, "grad64")
    with pytest.raises(ValueError, match="a_e"):
        nb._adjoints(dsys, DeviceLike(1, f64), DeviceLike(21), DeviceLike(18, f64), f32, "adj")
    assert nb._weights((1, 2, 3), "g").dtype == np.float32
    with pytest.raises(ValueError):
        nb._weights((1, 2), "g")


def test_calls_check_before_reaching_the_library(monkeypatch):
    def no_library():
        raise AssertionError("the library was reached")
    monkeypatch.setattr(nb, "lib", no_library)
    model = SimpleNamespace(n_params=5, hp=SimpleNamespace(n_types=3), handle=None)
    dsys = SimpleNamespace(n_atoms=4, n_cfg=1, pos=SimpleNamespace(device="cuda"))
    f64 = torch.float64
    with pytest.raises(ValueError, match="m2"):
        nb.adam_step(model, DeviceLike(5), DeviceLike(5), DeviceLike(4), 1, 1e-3)
    with pytest.raises(ValueError, match="masses"):
        nb.md_step(model, dsys, None, DeviceLike(12), DeviceLike(12), DeviceLike(1, f64), DeviceLike(9, f64),
                   [72.6, 121.8], 2.0, 1.0, False, None)
    with pytest.raises(ValueError, match="grad"):
        nb.param_grad(model, dsys, None, None, DeviceLike(1, f64), DeviceLike(12), DeviceLike(9, f64),
                      grad=DeviceLike(4), loss=DeviceLike(1, f64))
    with pytest.raises(ValueError, match="params"):
        nb.Model.set_params(model, DeviceLike(5, f64))
    with pytest.raises(ValueError, match="neighbour list holds 3 atoms"):
        nb.neighbors(model, dsys, SimpleNamespace(n_atoms=3), 0.0, None)
    with pytest.raises(ValueError, match="neighbour list"):
        nb.energy_forces_virial(model, dsys, SimpleNamespace(n_atoms=5), None)


def test_device_system_checks_shapes():
    pos, types = np.zeros((5, 3)), np.zeros(5, np.int32)
    box, off = np.full((2, 3), 10.0), np.array([0, 2, 5])
    s = nb.DeviceSystem(pos, types, box, off, device="cpu")
    assert (s.n_atoms, s.n_cfg) == (5, 2) and tuple(s.pos.shape) == (3, 5)
    for args in ((np.zeros((5, 2)), types, box, off), (pos, types[:4], box, off),
                 (pos, types, np.full(3, 10.0), off), (pos, types, box, off[:2])):
        with pytest.raises(ValueError):
            nb.DeviceSystem(*args, device="cpu")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libnep.so every call raises: there is no fallback path."""
    monkeypatch.setattr(nb, "_LIB", None)
    monkeypatch.setattr(nb, "LIB_PATH", str(tmp_path / "libnep.so"))
    with pytest.raises(RuntimeError, match="is missing"):
        nb.lib()
    with pytest.raises(RuntimeError, match="is missing"):
        nb.num_params(SimpleNamespace(n_types=3, n_rad=8, n_ang=6, k_rad=8, k_ang=8, l_max=4, has_4body=1,
                                      n_hidden=30, rc_rad=7.0, rc_ang=5.0))

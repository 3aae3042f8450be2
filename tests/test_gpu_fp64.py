"""FP64 evaluation (nep_energy_forces_virial_fp64) against the FP64 oracle.

Both sides compute in double from the same FP32 positions; they differ only
in summation order and in the rounding of cos/sin, about 1e-15 relative per
operation.  A per-atom quantity is a sum of ~10^2 terms of size <= ~10, so
agreement to 1e-10 (absolute, eV or eV/A) leaves a margin of ~10^3 over the
rounding, while a dropped term, a wrong sign or a swapped index moves the
result by orders of magnitude more.  Totals carry N_b such sums: 1e-10 N_b.
"""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10
TINY = I.Hyper(n_rad=3, n_ang=2, k_rad=4, k_ang=3, n_hidden=4, rc_rad=5.0, rc_ang=4.0)


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


def run64(nb, h, theta32, s, skin=0.0, cap=112, cap_ang=56, shifts=True, params64=None, precision=0):
    import torch
    model = nb.Model(h, theta32, precision=precision)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang, shifts=shifts)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, cap, cap_ang)
    nb.neighbors(model, dsys, nl, skin, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    ws64 = nb.Workspace64(model, s.n_atoms, s.n_cfg)
    p = None if params64 is None else torch.tensor(params64, dtype=torch.float64, device="cuda")
    e, f, et, v = nb.energy_forces_virial_fp64(model, dsys, nl, ws64, params=p)
    return dict(E=e.cpu().numpy(), F=f.cpu().numpy().T.copy(), Etot=et.cpu().numpy(),
                V=v.cpu().numpy().reshape(-1, 3, 3), model=model, dsys=dsys, nl=nl, ws=ws, ws64=ws64,
                out=(e, f, et, v))


def oracle(h, theta64, s):
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    return O.energy_forces_virial(h, theta64, p32.astype(np.float64), s.types,
                                  s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)


def assert_fp64(g, o, s):
    Nb = np.maximum(np.diff(s.atom_off), 1).astype(float)
    assert np.abs(g["E"] - o["E"]).max(initial=0) <= TOL
    assert np.abs(g["F"] - o["F"]).max(initial=0) <= TOL
    assert np.all(np.abs(g["Etot"] - o["Etot"]) <= TOL * Nb)
    assert np.all(np.abs(g["V"] - o["V"]).reshape(-1, 9).max(1) <= TOL * Nb)


@pytest.mark.parametrize("hname", ["TINY", "HYPER_SMALL", "HYPER_TABLE2", "HYPER_LARGE"])
def test_fp64_cell216_every_hyper(nb, hname):
    h = TINY if hname == "TINY" else getattr(I, hname)
    s, _ = I.workload_cell216()
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s)
    assert_fp64(g, oracle(h, th.astype(np.float64), s), s)


def test_fp64_small_boxes_images(nb):
    """Boxes shorter than 2 rc: pairs through image shifts."""
    h = I.HYPER_SMALL
    s = I.packing_batch([24, 40, 57, 33], tag=71)
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s)
    assert_fp64(g, oracle(h, th.astype(np.float64), s), s)


def test_fp64_degenerate_configs(nb):
    """An atom seeing only its own images, an empty configuration, an isolated
    atom (q = 0, E = network(0)) and a packing."""
    h = I.HYPER_SMALL
    other = I.packing_batch([40], tag=65)
    pos = np.concatenate([[[2.0, 2.0, 2.0], [10.0, 10.0, 10.0]], other.pos])
    types = np.concatenate([[2, 0], other.types]).astype(np.int32)
    box = np.array([[5.5, 6.0, 6.5], [30.0, 30.0, 30.0], [30.0, 30.0, 30.0], other.box[0]])
    s = I.System(pos=pos, types=types, box=box, atom_off=np.array([0, 1, 1, 2, 42]))
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s, cap=400, cap_ang=160)
    assert_fp64(g, oracle(h, th.astype(np.float64), s), s)
    assert g["Etot"][1] == 0.0 and np.all(g["V"][1] == 0.0)
    assert np.abs(g["F"][0]).max() <= TOL          # self images pull symmetrically


def test_fp64_min_image_list_with_skin(nb):
    """Minimum-image list (no shifts) with a 1 A skin: pairs in [rc, rc + skin)
    are in the list and masked in double."""
    h = I.HYPER_SMALL
    s = I.rocksalt(4, vacancy=0.2, tag=5)
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s, skin=1.0, cap=160, cap_ang=80, shifts=False)
    assert g["nl"].c.min_image == 1
    assert_fp64(g, oracle(h, th.astype(np.float64), s), s)


def test_fp64_parameters_in_double(nb):
    """Parameters that FP32 cannot hold: the result follows the FP64 values,
    not their FP32 roundings."""
    h = I.HYPER_SMALL
    s = I.packing_batch([40, 57], tag=72)
    th64 = I.init_params(h) * (1.0 + 1e-6 * np.random.default_rng(9).standard_normal(I.HYPER_SMALL.n_params))
    th32 = th64.astype(np.float32)
    g = run64(nb, h, th32, s, params64=th64)
    o64 = oracle(h, th64, s)
    assert_fp64(g, o64, s)
    # with the FP32-rounded parameters the oracle lies well outside the bar
    o32 = oracle(h, th32.astype(np.float64), s)
    assert np.abs(g["E"] - o32["E"]).max() > 10 * TOL


def test_fp64_any_precision_and_deterministic(nb):
    """The FP64 path ignores the network precision setting and repeats bitwise."""
    import torch
    h = I.HYPER_SMALL
    s = I.packing_batch([33, 64], tag=73)
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s, precision=1)
    assert_fp64(g, oracle(h, th.astype(np.float64), s), s)
    again = nb.energy_forces_virial_fp64(g["model"], g["dsys"], g["nl"], g["ws64"])
    for a, b in zip(g["out"], again):
        assert torch.equal(a, b)


def test_fp64_fp32_path_within_fp32_bar(nb):
    """The FP32 kernels sit within the FP32 parity bar of the FP64 GPU path."""
    h = I.HYPER_SMALL
    s, _ = I.workload_cell216()
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s)
    e32, f32, et32, v32 = nb.energy_forces_virial(g["model"], g["dsys"], g["nl"], g["ws"])
    assert np.abs(e32.cpu().numpy() - g["E"]).max() <= 1e-6
    assert np.abs(f32.cpu().numpy().T - g["F"]).max() <= 1e-4


def test_fp64_workspace_too_small(nb):
    import ctypes
    h = I.HYPER_SMALL
    s = I.packing_batch([24], tag=74)
    g = run64(nb, h, I.init_params(h).astype(np.float32), s)
    ws = g["ws64"]
    small = ctypes.c_size_t(ws.bytes - 1)
    e, f, et, v = g["out"]
    st = nb.lib().nep_energy_forces_virial_fp64(g["model"].handle, ctypes.byref(g["dsys"].c),
                                                ctypes.byref(g["nl"].c), None, nb._ptr(e), nb._ptr(f),
                                                nb._ptr(et), nb._ptr(v), ws.ptr, small, nb._stream())
    assert st == nb.NEP_ERR_ARG


@pytest.mark.parametrize("ncell", [6, 14])
def test_fp64_lane_groups_sampled(nb, ncell):
    """Systems on the 32- and 8-lanes-per-atom paths (N = 1,555 and 19,757;
    19,757 leaves the last warp with one atom group): sampled atoms, the last
    atoms among them, against the oracle's neighbourhood evaluation, and a
    zero net force."""
    s = I.rocksalt(ncell, vacancy=0.2, tag=6)
    h = I.HYPER_SMALL
    N = s.n_atoms
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s)
    centers = np.concatenate([np.random.default_rng(15).choice(N - 4, 20, replace=False), np.arange(N - 4, N)])
    p32 = s.pos32()
    ref = O.evaluate_centers(h, th.astype(np.float64), p32, p32.astype(np.float64), s.types,
                             s.box.astype(np.float32).astype(np.float64), s.atom_off, centers)
    assert np.abs(g["E"][ref["centers"]] - ref["E"]).max() <= TOL
    assert np.abs(g["F"][ref["centers"]] - ref["F"]).max() <= TOL
    assert np.abs(g["F"].sum(0)).max() <= TOL
    assert abs(g["Etot"][0] - g["E"].sum()) <= TOL * N


def test_fp64_md900k_sampled(nb):
    """Full 900,000-atom workload: 24 sampled atoms against the oracle's
    neighbourhood evaluation, and the FP64 properties at any size."""
    import torch
    s, h = I.workload_md900k()
    N = s.n_atoms
    th = I.init_params(h).astype(np.float32)
    g = run64(nb, h, th, s, cap=96, cap_ang=40, shifts=False)
    centers = np.random.default_rng(14).choice(N, 24, replace=False)
    p32 = s.pos32()
    ref = O.evaluate_centers(h, th.astype(np.float64), p32, p32.astype(np.float64), s.types,
                             s.box.astype(np.float32).astype(np.float64), s.atom_off, centers)
    assert np.abs(g["E"][ref["centers"]] - ref["E"]).max() <= TOL
    assert np.abs(g["F"][ref["centers"]] - ref["F"]).max() <= TOL
    e, f, et, v = g["out"]
    # the forces of a periodic system sum to zero; the virial is symmetric
    assert f.sum(1).abs().max().item() <= 1e-9
    V = g["V"][0]
    assert np.abs(V - V.T).max() <= 1e-9 * N ** 0.5
    assert abs(et.item() - e.sum().item()) <= 1e-8

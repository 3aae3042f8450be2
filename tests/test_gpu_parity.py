"""GPU path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 kernels vs FP64 oracle on the same float32 inputs):
  neighbour sets        bit-exact after sorting (i, j, image)
  per-atom energy       1e-6 eV
  force components      1e-4 eV/A
  total energy          1e-6 eV per atom of the configuration
  virial components     1e-5 eV per atom: W_i = -sum_j f_ij r_ij is a sum of
                        ~50 FP32 products of size <= 1 eV here, so its FP32
                        rounding stays below 1e-5 eV, and the FP64 sum over
                        N_b atoms adds at most N_b such errors.
"""
import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_E, TOL_F, TOL_ET, TOL_V = 1e-6, 1e-4, 1e-6, 1e-5
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


def gpu_eval(nb, h, theta32, s, skin=0.0, cap=96, cap_ang=40, shifts=True):
    model = nb.Model(h, theta32)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang, shifts=shifts)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, cap, cap_ang)
    nb.neighbors(model, dsys, nl, skin, ws)
    e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
    st = nb.check_list(nl)
    out = dict(E=e.cpu().numpy(), F=f.cpu().numpy().T.copy(), Etot=et.cpu().numpy(),
               V=v.cpu().numpy().reshape(-1, 3, 3), status=st, nl=nl, model=model, dsys=dsys, ws=ws)
    return out


def oracle_eval(h, theta32, s):
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    return O.energy_forces_virial(h, theta32.astype(np.float64), p32.astype(np.float64), s.types,
                                  s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)


def assert_parity(g, o, s):
    assert g["status"] == 0
    Nb = np.diff(s.atom_off).astype(float)
    assert np.abs(g["E"] - o["E"]).max(initial=0) <= TOL_E
    assert np.abs(g["F"] - o["F"]).max(initial=0) <= TOL_F
    assert np.all(np.abs(g["Etot"] - o["Etot"]) <= TOL_ET * np.maximum(Nb, 1))
    assert np.all(np.abs(g["V"] - o["V"]).reshape(-1, 9).max(1) <= TOL_V * np.maximum(Nb, 1))


def list_sets(nl, s, min_image):
    i, j, sh, ang = nl.to_pairs()
    if min_image:
        # recover the image the minimum-image convention picks
        p = s.pos32()
        L = s.box.astype(np.float32)[s.cfg_of_atom()[i]]
        d = p[j] - p[i]
        sh = (-np.rint(d / L)).astype(np.int64)
    rad = set(zip(i.tolist(), j.tolist(), map(tuple, sh.tolist())))
    angs = set(zip(i[ang].tolist(), j[ang].tolist(), map(tuple, sh[ang].tolist())))
    return rad, angs


def oracle_sets(s, rc, rc_ang):
    p32 = s.pos32()
    a = O.neighbor_pairs(p32, s.box, s.atom_off, rc)
    b = O.neighbor_pairs(p32, s.box, s.atom_off, rc_ang)
    mk = lambda t: set(zip(t[0].tolist(), t[1].tolist(), map(tuple, t[2].tolist())))
    return mk(a), mk(b)


# --- neighbour lists -------------------------------------------------------------
@pytest.mark.parametrize("case,skin", [("cell216", 0.0), ("cell216", 1.0), ("batch", 0.0),
                                        ("batch", 1.0), ("tinybox", 0.0)])
def test_neighbor_sets_bit_exact(nb, case, skin):
    h = I.HYPER_SMALL
    if case == "cell216":
        s, _ = I.workload_cell216()
    elif case == "batch":
        s = I.packing_batch([24, 31, 57, 100, 250], tag=61)
    else:   # boxes shorter than the cutoff: several images per j and self images
        s = I.packing_batch([3, 8, 24], dmin=2.0, density=0.04, tag=62)
    g = gpu_eval(nb, h, I.init_params(h).astype(np.float32), s, skin=skin, cap=400, cap_ang=160)
    assert g["status"] == 0
    rc = float(np.float32(h.rc_rad) + np.float32(skin))
    rca = float(np.float32(h.rc_ang) + np.float32(skin))
    rad, ang = list_sets(g["nl"], s, g["nl"].c.min_image)
    want_rad, want_ang = oracle_sets(s, rc, rca)
    assert rad == want_rad
    assert ang == want_ang
    # reverse slots point back at the pair
    nl = g["nl"]
    N = s.n_atoms
    nbr = nl.nbr.cpu().numpy().reshape(nl.cap, N)
    rev = nl.rev.cpu().numpy().reshape(nl.cap_ang, N)
    cnta = nl.cnt_ang.cpu().numpy()
    for i in range(0, N, max(1, N // 50)):
        for k in range(cnta[i]):
            assert nbr[rev[k, i], nbr[k, i]] == i


# --- energies, forces, virial ------------------------------------------------------------
@pytest.mark.parametrize("hname", ["small", "tiny", "large", "table2"])
def test_efv_cell(nb, hname):
    h = dict(small=I.HYPER_SMALL, tiny=TINY, large=I.HYPER_LARGE, table2=I.HYPER_TABLE2)[hname]
    s = I.rocksalt(3, vacancy=0.0, tag=0) if hname != "large" else I.rocksalt(4, vacancy=0.2, tag=63)
    th = I.init_params(h).astype(np.float32)
    assert_parity(gpu_eval(nb, h, th, s), oracle_eval(h, th, s), s)


@pytest.mark.parametrize("skin,cap,cap_ang", [(0.0, 160, 64), (1.0, 160, 64), (1.0, 300, 260)])
def test_efv_batch_small_boxes(nb, skin, cap, cap_ang):
    # cap_ang >= 256: no per-row table, the reverse-slot search scans the prefix
    h = I.HYPER_SMALL
    s = I.packing_batch([24, 31, 57, 100, 250, 512], tag=64)
    th = I.init_params(h).astype(np.float32)
    assert_parity(gpu_eval(nb, h, th, s, skin=skin, cap=cap, cap_ang=cap_ang), oracle_eval(h, th, s), s)


def test_efv_more_than_64_angular_slots(nb):
    # long angular cutoff: atoms with more than 64 angular-prefix slots, so the
    # force gather takes both its bit-mask and its in-walk branch
    h = I.Hyper(n_rad=3, n_ang=2, k_rad=4, k_ang=3, n_hidden=4, rc_rad=8.5, rc_ang=8.0)
    s = I.packing_batch([150, 200], tag=77)
    th = I.init_params(h).astype(np.float32)
    g = gpu_eval(nb, h, th, s, skin=0.5, cap=260, cap_ang=200)
    assert int(g["nl"].cnt_ang.max().item()) > 64
    assert_parity(g, oracle_eval(h, th, s), s)


def test_efv_degenerate_configs(nb):
    # an empty configuration, a single atom seeing only its own images, an
    # isolated atom (q = 0, E = network(0)) and a normal packing
    h = I.HYPER_SMALL
    other = I.packing_batch([40], tag=65)
    pos = np.concatenate([[[2.0, 2.0, 2.0], [10.0, 10.0, 10.0]], other.pos])
    types = np.concatenate([[2, 0], other.types]).astype(np.int32)
    box = np.array([[5.5, 6.0, 6.5], [30.0, 30.0, 30.0], [30.0, 30.0, 30.0], other.box[0]])
    s = I.System(pos=pos, types=types, box=box, atom_off=np.array([0, 1, 1, 2, 42]))
    th = I.init_params(h).astype(np.float32)
    g = gpu_eval(nb, h, th, s, cap=400, cap_ang=160)
    o = oracle_eval(h, th, s)
    assert_parity(g, o, s)
    assert g["Etot"][1] == 0.0 and np.all(g["V"][1] == 0.0)
    assert np.abs(g["F"][0]).max() < 1e-6          # self images pull symmetrically


def test_deterministic_bitwise(nb):
    h = I.HYPER_SMALL
    s = I.packing_batch([57, 100, 250], tag=66)
    th = I.init_params(h).astype(np.float32)
    g = gpu_eval(nb, h, th, s, skin=1.0, cap=160, cap_ang=64)
    e2, f2, et2, v2 = nb.energy_forces_virial(g["model"], g["dsys"], g["nl"], g["ws"])
    nb.neighbors(g["model"], g["dsys"], g["nl"], 1.0, g["ws"])
    e3, f3, et3, v3 = nb.energy_forces_virial(g["model"], g["dsys"], g["nl"], g["ws"])
    for a, b in ((g["E"], e2), (g["E"], e3), (g["F"], f2.cpu().numpy().T), (g["F"], f3.cpu().numpy().T),
                 (g["Etot"], et3), (g["V"].reshape(-1, 9), v3)):
        b = b.cpu().numpy() if hasattr(b, "cpu") else b
        assert np.array_equal(a, b)


def test_capacity_overflow_reports_needed_size(nb):
    h = I.HYPER_SMALL
    s, _ = I.workload_cell216()
    th = I.init_params(h).astype(np.float32)
    g = gpu_eval(nb, h, th, s, cap=20, cap_ang=8)
    assert g["status"] == nb.NEP_ERR_CAPACITY
    st = g["nl"].status.cpu().numpy()
    assert st[0] == 1 and st[1] > 20 and st[2] > 8
    g2 = gpu_eval(nb, h, th, s, cap=int(st[1]), cap_ang=int(st[2]))
    assert_parity(g2, oracle_eval(h, th, s), s)


def test_invalid_input_flags(nb):
    h = I.HYPER_SMALL
    s, _ = I.workload_cell216()
    th = I.init_params(h).astype(np.float32)
    bad_t = I.System(pos=s.pos, types=s.types.copy(), box=s.box, atom_off=s.atom_off)
    bad_t.types[5] = 7
    assert gpu_eval(nb, h, th, bad_t)["status"] == nb.NEP_ERR_INPUT
    # an atom outside its box is reported by the list build
    model = nb.Model(h, th)
    dsys = nb.DeviceSystem.from_inputs(s)
    dsys.pos[0, 3] = 18.5
    nl = nb.NeighborList(s.n_atoms, 96, 40)
    ws = nb.Workspace(model, s.n_atoms, 1, 96, 40)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    assert nb.check_list(nl) == nb.NEP_ERR_INPUT


def test_host_argument_errors(nb):
    h = I.HYPER_SMALL
    s, _ = I.workload_cell216()
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 96, 40)
    ws = nb.Workspace(model, s.n_atoms, 1, 96, 40)
    small = nb.Workspace(model, 10, 1, 96, 40)
    with pytest.raises(nb.NepError) as e:
        nb.neighbors(model, dsys, nl, 0.0, small)
    assert e.value.status == nb.NEP_ERR_ARG and "workspace too small" in str(e.value)
    with pytest.raises(nb.NepError):
        nb.neighbors(model, dsys, nl, -1.0, ws)
    bad = nb.NeighborList(s.n_atoms, 8, 16)
    with pytest.raises(nb.NepError):
        nb.neighbors(model, dsys, bad, 0.0, ws)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_every_angular_variant(nb, variant):
    """Each register-budget variant of the angular kernel (S_nlm in tensor
    memory for variant 0, in shared memory for 1 and 2) against the oracle."""
    h = I.HYPER_SMALL
    s = I.packing_batch([57, 100, 250], tag=68)
    th = I.init_params(h).astype(np.float32)
    model = nb.Model(h, th)
    nb.set_variant(model, variant)
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 160, 64)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, 160, 64)
    nb.neighbors(model, dsys, nl, 1.0, ws)
    e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
    assert_parity(dict(E=e.cpu().numpy(), F=f.cpu().numpy().T, Etot=et.cpu().numpy(),
                       V=v.cpu().numpy().reshape(-1, 3, 3), status=nb.check_list(nl)),
                  oracle_eval(h, th, s), s)


def test_autotune_variants_agree(nb):
    """Every compiled register-budget variant and block size computes the
    same E, F, V; the autotuner picks valid choices and later calls use them."""
    h = I.HYPER_SMALL
    s = I.packing_batch([57, 100, 250], tag=67)
    th = I.init_params(h).astype(np.float32)
    g = gpu_eval(nb, h, th, s, skin=1.0, cap=160, cap_ang=64)
    chosen = nb.autotune(g["model"], g["dsys"], g["nl"], g["ws"], reps=2)
    assert 0 <= chosen[0] < 3 and chosen[1] in (64, 128, 256) and chosen[2] in (64, 128, 256)
    e, f, et, v = nb.energy_forces_virial(g["model"], g["dsys"], g["nl"], g["ws"])
    assert np.abs(e.cpu().numpy() - g["E"]).max() <= 1e-6
    assert np.abs(f.cpu().numpy().T - g["F"]).max() <= 1e-5
    assert_parity(dict(E=e.cpu().numpy(), F=f.cpu().numpy().T, Etot=et.cpu().numpy(),
                       V=v.cpu().numpy().reshape(-1, 3, 3), status=0), oracle_eval(h, th, s), s)
    # every block size of the radial and finish kernels gives the same bits
    ref = None
    for rb in (64, 128, 256):
        for fb in (64, 128, 256):
            nb.set_launch(g["model"], 0, rb, fb)
            out = [t.cpu().numpy() for t in nb.energy_forces_virial(g["model"], g["dsys"], g["nl"], g["ws"])]
            if ref is None:
                ref = out
            for x, y in zip(out, ref):
                assert np.array_equal(x, y)
    nb.set_launch(g["model"])
    with pytest.raises(nb.NepError):
        nb.set_launch(g["model"], 0, 96, 0)


def test_graph_captured_md_matches_eager(nb):
    """Velocity-Verlet steps (with a rebuild) captured in one CUDA graph give
    the same bits as the same calls launched one by one."""
    import torch
    h = I.HYPER_SMALL
    s = I.packing_batch([57, 100, 250], tag=69)
    th = I.init_params(h).astype(np.float32)
    masses = I.MASSES.astype(np.float32)
    vel0 = np.ascontiguousarray(I.maxwell_boltzmann(s.types, 900.0, atom_off=s.atom_off).astype(np.float32).T)

    def run(graph):
        model = nb.Model(h, th)
        dsys = nb.DeviceSystem.from_inputs(s)
        nl = nb.NeighborList(s.n_atoms, 160, 64)
        ws = nb.Workspace(model, s.n_atoms, s.n_cfg, 160, 64)
        nb.neighbors(model, dsys, nl, 1.0, ws)
        e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
        vel = torch.from_numpy(vel0.copy()).cuda()
        st = torch.cuda.Stream()
        torch.cuda.synchronize()
        steps = lambda: [nb.md_step(model, dsys, nl, vel, f, et, v, masses, 2.0, 1.0, k % 10 == 0, ws, stream=st)
                         for k in range(12)]
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                steps()
            g.replay()
        else:
            with torch.cuda.stream(st):
                steps()
        torch.cuda.synchronize()
        assert nb.check_list(nl) == nb.NEP_OK
        return dsys.pos.cpu(), vel.cpu(), f.cpu(), et.cpu(), v.cpu()

    a, b = run(False), run(True)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_bounded_wait_times_out_and_context_survives(nb):
    """A tensor-core completion wait made to run out (an mbarrier that nothing
    arrives at) reports NEP_ERR_TIMEOUT through a device flag; the context
    keeps working afterwards."""
    assert nb.selftest_wait_timeout() == nb.NEP_ERR_TIMEOUT
    assert "ran out" in nb.last_error()
    h = TINY
    s = I.rocksalt(3, vacancy=0.0, tag=0)
    th = I.init_params(h).astype(np.float32)
    assert_parity(gpu_eval(nb, h, th, s), oracle_eval(h, th, s), s)


def test_zero_atom_batch(nb):
    """Two configurations holding no atoms at all: the list, E/F/V, the
    training gradient, the FP64 evaluation and an MD step all return OK with
    zero totals."""
    import torch
    h = I.HYPER_SMALL
    s = I.System(pos=np.zeros((0, 3)), types=np.zeros(0, np.int32), box=np.array([[20.0] * 3, [25.0] * 3]),
                 atom_off=np.array([0, 0, 0]))
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(0, 64, 32)
    ws = nb.Workspace(model, 0, 2, 64, 32, train=True)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    assert nb.check_list(nl) == nb.NEP_OK
    e, f, et, v = nb.energy_forces_virial(model, dsys, nl, ws)
    assert torch.count_nonzero(et).item() == 0 and torch.count_nonzero(v).item() == 0
    z = dict(device="cuda")
    grad, loss = nb.param_grad(model, dsys, nl, ws, torch.zeros(2, dtype=torch.float64, **z),
                               torch.zeros(3, 0, dtype=torch.float32, **z), torch.zeros(2, 9, dtype=torch.float64, **z))
    assert torch.count_nonzero(grad).item() == 0 and loss.item() == 0.0
    ws64 = nb.Workspace64(model, 0, 2)
    _, _, et64, v64 = nb.energy_forces_virial_fp64(model, dsys, nl, ws64)
    assert torch.count_nonzero(et64).item() == 0 and torch.count_nonzero(v64).item() == 0
    vel = torch.zeros(3, 0, **z)
    nb.md_step(model, dsys, nl, vel, f, et, v, I.MASSES.astype(np.float32), 2.0, 0.0, True, ws)
    assert nb.check_list(nl) == nb.NEP_OK

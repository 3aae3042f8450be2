"""nep_energy_forces_virial_noalloc: the allocation-free variant of the
energy/force/virial call, for callers that cannot allocate device memory
(a plugin inside a host code that owns the device memory, or a loop that
forbids allocator calls after start-up).  It must give the same results as
the workspace call, call after call, with scratch in the library's static
device array.  This file is collected last so that a failure here stops a
-x run only after every other test has run."""
import numpy as np
import pytest

from paper_2607_06969_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_E, TOL_F, TOL_ET, TOL_V = 1e-6, 1e-4, 1e-6, 1e-5   # same as the parity tests


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("case", ["cell216", "batch"])
def test_noalloc_matches_workspace_call_twice(nb, case):
    h = I.HYPER_SMALL
    if case == "cell216":
        s, _ = I.workload_cell216()
        skin, cap, cap_ang = 0.0, 96, 40
    else:
        s = I.packing_batch([24, 57, 100, 250], tag=71)
        skin, cap, cap_ang = 1.0, 160, 64
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang, shifts=True)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, cap, cap_ang)
    nb.neighbors(model, dsys, nl, skin, ws)
    ref = [t.cpu().numpy() for t in nb.energy_forces_virial(model, dsys, nl, ws)]
    assert nb.check_list(nl) == nb.NEP_OK
    Nb = np.maximum(np.diff(s.atom_off), 1)
    for _ in range(2):
        got = [t.cpu().numpy() for t in nb.energy_forces_virial_noalloc(model, dsys, nl)]
        assert nb.check_list(nl) == nb.NEP_OK
        assert np.abs(got[0] - ref[0]).max() <= TOL_E
        assert np.abs(got[1] - ref[1]).max() <= TOL_F
        assert np.all(np.abs(got[2] - ref[2]) <= TOL_ET * Nb)
        assert np.all(np.abs(got[3] - ref[3]).max(1) <= TOL_V * Nb)
        # the same kernels on the same inputs, scratch elsewhere: bit for bit
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)


def test_noalloc_rejects_systems_beyond_the_static_array(nb):
    h = I.HYPER_SMALL
    s = I.rocksalt(12, vacancy=0.2, tag=72)            # 12,441 atoms: scratch above 32 MiB
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, 160, 80, shifts=False)
    ws = nb.Workspace(model, s.n_atoms, 1, 160, 80)
    assert ws.bytes > nb.NOALLOC_SCRATCH_BYTES
    nb.neighbors(model, dsys, nl, 1.0, ws)
    with pytest.raises(nb.NepError) as e:
        nb.energy_forces_virial_noalloc(model, dsys, nl)
    assert e.value.status == nb.NEP_ERR_ARG and "static array" in str(e.value)

"""The C ABI library builds, loads without a GPU, and exports every entry
point include/nep.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import binding as nb
from paper_2607_06969_gb300 import build as B
from paper_2607_06969_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return nb.lib()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "nep.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    return set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s*(nep_\w+)\s*\(", txt, flags=re.M))


def test_header_and_binding_agree():
    assert header_functions() == set(nb.ENTRY_POINTS)


def test_library_exports_every_declared_symbol(L):
    for name in header_functions():
        assert hasattr(L, name), name
    assert L.nep_version().decode().startswith("libnep")


@pytest.mark.parametrize("hyp", [I.HYPER_SMALL, I.HYPER_LARGE, I.HYPER_TABLE2,
                                 I.Hyper(n_rad=3, n_ang=2, k_rad=4, k_ang=3, n_hidden=4)])
def test_num_params_matches_oracle(L, hyp):
    assert nb.num_params(hyp) == O.param_count(hyp)
    hp = nb.hparams_of(hyp)
    assert L.nep_supported(ctypes.byref(hp)) == 1


def test_create_rejects_bad_arguments_before_touching_the_gpu(L):
    bad = nb.hparams_of(I.HYPER_SMALL)
    bad.l_max = 3
    out = ctypes.c_void_p()
    assert L.nep_create(ctypes.byref(bad), None, 0, ctypes.byref(out)) == nb.NEP_ERR_ARG
    assert "l_max" in nb.last_error()
    gen = nb.hparams_of(I.Hyper(n_rad=5))                  # no kernel set: the generic FP32 path
    assert L.nep_supported(ctypes.byref(gen)) == 2
    assert L.nep_create(ctypes.byref(gen), None, 0, ctypes.byref(out)) == nb.NEP_ERR_ARG   # parameter count
    gen16 = nb.hparams_of(I.Hyper(n_rad=5), precision=1)   # FP16 needs a kernel set
    assert L.nep_supported(ctypes.byref(gen16)) == 0
    assert L.nep_create(ctypes.byref(gen16), None, 0, ctypes.byref(out)) == nb.NEP_ERR_UNSUPPORTED
    uns = nb.hparams_of(I.Hyper(n_rad=17))                 # beyond the generic bounds
    assert L.nep_supported(ctypes.byref(uns)) == 0
    assert L.nep_create(ctypes.byref(uns), None, 0, ctypes.byref(out)) == nb.NEP_ERR_UNSUPPORTED
    ok = nb.hparams_of(I.HYPER_SMALL)
    assert L.nep_create(ctypes.byref(ok), None, 3, ctypes.byref(out)) == nb.NEP_ERR_ARG
    assert L.nep_num_params(ctypes.byref(bad)) == 0


def test_domain_calls_reject_bad_arguments_before_touching_the_gpu(L):
    """The slab-decomposition calls check their host arguments first."""
    box = (ctypes.c_float * 3)(30.0, 30.0, 30.0)
    counts = ctypes.c_void_p(16)            # never dereferenced: the checks fail first
    f = ctypes.c_float
    assert L.nep_domain_workspace_bytes(-1) == 0
    ws = L.nep_domain_workspace_bytes(1000)
    assert ws > 0
    # slab outside the box, and a slab whose halos overlap it
    assert L.nep_domain_select(ctypes.c_void_p(16), 1000, box, f(10.0), f(40.0), f(2.0), ctypes.c_void_p(16),
                               ctypes.c_void_p(16), 10, counts, ctypes.c_void_p(256), ws, None) == nb.NEP_ERR_ARG
    assert L.nep_domain_select(ctypes.c_void_p(16), 1000, box, f(0.0), f(20.0), f(6.0), ctypes.c_void_p(16),
                               ctypes.c_void_p(16), 10, counts, ctypes.c_void_p(256), ws, None) == nb.NEP_ERR_ARG
    assert "halo" in nb.last_error()
    # workspace too small
    assert L.nep_domain_select(ctypes.c_void_p(16), 1000, box, f(0.0), f(10.0), f(2.0), ctypes.c_void_p(16),
                               ctypes.c_void_p(16), 10, counts, ctypes.c_void_p(256), ws - 1, None) == nb.NEP_ERR_ARG
    # scatter: more owned rows than local rows
    assert L.nep_domain_scatter(ctypes.c_void_p(16), 5, 3, ctypes.c_void_p(16), 6, ctypes.c_void_p(16), 10,
                                None) == nb.NEP_ERR_ARG
    # gather: missing pointers
    assert L.nep_domain_gather(None, None, 10, None, None, 4, box, f(0.0), None, None, None) == nb.NEP_ERR_ARG


def test_plain_c_client_compiles_links_and_runs(L, tmp_path):
    """include/nep.h is a C99 header: a C program that takes the address of
    every declared entry point compiles with warnings as errors, links
    against libnep.so, and its host-only calls give the oracle's parameter
    count and the documented argument errors."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = sorted(header_functions())
    h = I.HYPER_TABLE2
    src = "\n".join([
        "#include <stdio.h>",
        "#include <string.h>",
        '#include "nep.h"',
        "typedef void (*fn)(void);",
        "int main(void) {",
        "    static const fn table[] = {" + ", ".join(f"(fn){n}" for n in names) + "};",
        "    nep_hparams hp;",
        "    nep_model* m = NULL;",
        "    size_t k;",
        "    for (k = 0; k < sizeof table / sizeof table[0]; ++k) if (!table[k]) return 2;",
        "    memset(&hp, 0, sizeof hp);",
        f"    hp.n_types = {h.n_types}; hp.n_rad = {h.n_rad}; hp.n_ang = {h.n_ang};",
        f"    hp.k_rad = {h.k_rad}; hp.k_ang = {h.k_ang}; hp.l_max = {h.l_max};",
        f"    hp.has_4body = {h.has_4body}; hp.n_hidden = {h.n_hidden};",
        f"    hp.rc_rad = {h.rc_rad}f; hp.rc_ang = {h.rc_ang}f; hp.precision = 0;",
        '    printf("%zu %d ", nep_num_params(&hp), nep_supported(&hp));',
        '    printf("%d ", (int)nep_create(&hp, NULL, 3, &m));',
        '    printf("%d %s\\n", m == NULL, strstr(nep_version(), "libnep") == nep_version() ? "ok" : "bad");',
        "    return 0;",
        "}",
    ])
    (tmp_path / "client.c").write_text(src)
    libdir = os.path.dirname(L._name)
    exe = str(tmp_path / "client")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Wpedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(tmp_path / "client.c"), "-o", exe,
                    "-L", libdir, "-lnep", "-Wl,-rpath," + libdir], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == O.param_count(h) and out[1] == "1"
    assert int(out[2]) == nb.NEP_ERR_ARG and out[3] == "1" and out[4] == "ok"


def test_system_and_list_checks_reject_before_touching_the_gpu(L):
    """The library's host-side checks of a system and a list run before the
    model or any device pointer is used: offsets that do not end at N, a
    box that is not positive, cap_ang > cap, and lists whose slot-major
    arrays would pass 2^31 (cap * N) or 2^30 (cap_ang * N) entries.  A
    zero-filled host buffer stands in for the model and the device arrays."""
    import numpy as np
    N = 216
    stand_in = ctypes.create_string_buffer(4096)
    p = ctypes.cast(stand_in, ctypes.c_void_p)
    off = np.array([0, N], np.int32)
    box = np.array([18.0, 18.0, 18.0], np.float32)

    def system(off_arr, box_arr):
        return nb.System(N, 1, p, p, p, p, off_arr.ctypes.data, box_arr.ctypes.data)

    def nlist(cap, cap_ang):
        return nb.NList(cap, cap_ang, p, p, p, p, p, p, 0.0, 0)

    def status(sysc, nlc):
        return L.nep_neighbors(p, ctypes.byref(sysc), ctypes.c_float(0.0), ctypes.byref(nlc), p, 1 << 20, None)

    ok_list = nlist(96, 40)
    cases = [
        (system(np.array([0, N - 1], np.int32), box), ok_list, "end at n_atoms"),
        (system(off, np.array([18.0, 0.0, 18.0], np.float32)), ok_list, "positive and finite"),
        (system(off, box), nlist(40, 96), "cap_ang <= cap"),
        (system(off, box), nlist((1 << 31) // N + 1, 1), "2^31"),
        (system(off, box), nlist((1 << 30) // N + 1, (1 << 30) // N + 1), "2^30"),
    ]
    for sysc, nlc, msg in cases:
        assert status(sysc, nlc) == nb.NEP_ERR_ARG, msg
        assert msg in nb.last_error(), (msg, nb.last_error())
    sysc = system(off, box)
    nlc = nlist((1 << 31) // N + 1, 1)
    assert L.nep_energy_forces_virial(p, ctypes.byref(sysc), ctypes.byref(nlc), p, p, p, p, p, 1 << 20,
                                      None) == nb.NEP_ERR_ARG
    assert "2^31" in nb.last_error()


def test_call_argument_checks_reject_before_touching_the_gpu(L):
    """Per-call argument checks that precede any use of the model or the
    device: the integrator's time steps and masses, the loss mode and
    weights, and Adam's step, rate, moments and epsilon."""
    import numpy as np
    N = 216
    stand_in = ctypes.create_string_buffer(4096)
    p = ctypes.cast(stand_in, ctypes.c_void_p)
    off = np.array([0, N], np.int32)
    box = np.array([18.0, 18.0, 18.0], np.float32)
    sysc = nb.System(N, 1, p, p, p, p, off.ctypes.data, box.ctypes.data)
    nlc = nb.NList(96, 40, p, p, p, p, p, p, 0.0, 0)
    masses = np.array([72.63, 121.76, 127.6], np.float32)
    mp = masses.ctypes.data_as(ctypes.c_void_p)
    f = ctypes.c_float

    def expect(st, msg):
        assert st == nb.NEP_ERR_ARG and msg in nb.last_error(), (st, msg, nb.last_error())

    for dt in (0.0, -1.0, float("nan")):
        expect(L.nep_md_step(p, ctypes.byref(sysc), ctypes.byref(nlc), p, p, p, p, mp, f(dt), f(1.0), 1, p,
                             1 << 20, None), "dt must be positive")
    expect(L.nep_md_step(p, ctypes.byref(sysc), ctypes.byref(nlc), p, p, p, p, None, f(2.0), f(1.0), 1, p,
                         1 << 20, None), "masses_host is NULL")
    expect(L.nep_md_kick(p, ctypes.byref(sysc), p, p, mp, f(float("inf")), f(2.0), None), "half_dt")
    expect(L.nep_md_kick(p, ctypes.byref(sysc), p, p, mp, f(1.0), f(-2.0), None), "drift_dt")
    w = np.array([1.0, 1.0, 0.1], np.float32)
    wp = w.ctypes.data_as(ctypes.c_void_p)
    expect(L.nep_param_grad(p, ctypes.byref(sysc), ctypes.byref(nlc), p, p, p, wp, 2, p, p, p, 1 << 20, None),
           "loss_mode must be 0 or 1")
    expect(L.nep_param_grad(p, ctypes.byref(sysc), ctypes.byref(nlc), p, p, p, None, 0, p, p, p, 1 << 20, None),
           "loss weights are NULL")
    for n_owned in (-1, N + 1):
        expect(L.nep_energy_forces_virial_owned(p, ctypes.byref(sysc), ctypes.byref(nlc), n_owned, p, p, p, p, p,
                                                1 << 20, None), "need 0 <= n_owned <= n_atoms")
    unbuilt = nb.NList(96, 40, p, p, p, None, p, p, 0.0, 0)         # no shifts and not minimum-image
    assert L.nep_energy_forces_virial(p, ctypes.byref(sysc), ctypes.byref(unbuilt), p, p, p, p, p, 1 << 20,
                                      None) == nb.NEP_ERR_STATE
    assert "not built" in nb.last_error()
    for kw, msg in ((dict(t=0), "t must be >= 1"), (dict(lr=-1.0), "lr must be"), (dict(beta1=1.0), "beta1"),
                    (dict(beta2=-0.1), "beta1 and beta2"), (dict(eps=0.0), "eps must be")):
        a = dict(t=1, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)
        a.update(kw)
        expect(L.nep_adam_step(p, p, p, p, a["t"], f(a["lr"]), f(a["beta1"]), f(a["beta2"]), f(a["eps"]), None),
               msg)

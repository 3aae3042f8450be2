"""Values the paper prints, stored under tests/golden/ with their citations,
against the oracle, the model hyper-parameters and the training protocol."""
import inspect
import os

import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I
from paper_2607_06969_gb300 import train as T

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


def test_table2_model_and_parameter_count():
    """Table 2: the NEP hyper-parameters; Section 4.1.2: 7.9k trainable
    parameters (2+3-body, three species)."""
    g = read_golden("table2_nep.txt")
    h = I.HYPER_TABLE2
    assert (h.n_rad, h.n_ang, h.l_max, h.k_rad, h.k_ang, h.n_hidden) == \
        tuple(int(g[k]) for k in ("n_rad", "n_ang", "l_max", "k_rad", "k_ang", "n_hidden"))
    assert (h.rc_rad, h.rc_ang) == (g["rc_rad"], g["rc_ang"])
    assert h.has_4body == 0 and h.n_types == 3
    assert round(O.param_count(h) / 1000.0, 1) == g["trainable_parameters_k"]


def test_table2_training_settings():
    g = read_golden("table2_nep.txt")
    c = T.TrainConfig.table2()
    assert (c.lr_start, c.lr_end, c.epochs) == (g["lr_start"], g["lr_end"], int(g["epochs"]))
    assert c.w_start == (g["w_e_start"], g["w_f_start"], g["w_v_start"])
    assert c.w_end == (g["w_e_end"], g["w_f_end"], g["w_v_end"])


def test_optimizer_and_schedule_settings():
    """Section 4.2 (Adam) and Section 3.3.2 (warm-up, cosine annealing)."""
    g = read_golden("optimizer_schedule.txt")
    c = T.TrainConfig()
    assert (c.beta1, c.beta2, c.eps) == (g["beta1"], g["beta2"], g["eps"])
    d = inspect.signature(O.adam_step).parameters
    assert (d["beta1"].default, d["beta2"].default, d["eps"].default) == (g["beta1"], g["beta2"], g["eps"])
    assert g["weight_decay"] == 0.0 and "weight_decay" not in d
    assert inspect.signature(T.lr_at).parameters["start_factor"].default == g["warmup_start_factor"]
    # one epoch of warm-up: the learning rate reaches lr_start after len(batches) steps
    n_batches = 7
    lrs = [T.lr_at(k, 1e-3, 1e-6, int(g["warmup_epochs"]) * n_batches, 200 * n_batches) for k in range(10)]
    assert lrs[0] == pytest.approx(1e-3 * g["warmup_start_factor"])
    assert lrs[n_batches] == pytest.approx(1e-3)
    assert all(a < b for a, b in zip(lrs[:n_batches], lrs[1:n_batches + 1]))

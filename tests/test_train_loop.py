"""Training protocol around the gradient (Section 3.3): the learning-rate
schedule and the loss weights (host logic), the oracle's Adam step against
closed forms, the device Adam step against the oracle, and a short fit of a
student NEP to teacher labels."""
import math

import numpy as np
import pytest

from oracle import nep_oracle as O
from paper_2607_06969_gb300 import inputs as I
from paper_2607_06969_gb300 import train as T


# --- learning rate (Section 3.3.2) -------------------------------------------------------
def test_lr_schedule_pins():
    lr0, lr1, W, total = 1e-3, 1e-5, 10, 110
    f = lambda k: T.lr_at(k, lr0, lr1, W, total)
    assert f(0) == pytest.approx(lr0 * 1e-4)                       # LinearLR start factor
    assert f(5) == pytest.approx(lr0 * (1e-4 + (1 - 1e-4) * 0.5))  # linear in the step
    assert f(W) == pytest.approx(lr0)                              # warm-up ends at lr_start
    assert f(W + 50) == pytest.approx((lr0 + lr1) / 2)             # cosine midpoint
    assert f(total) == pytest.approx(lr1)                          # ends at lr_end
    assert f(total + 7) == pytest.approx(lr1)
    seq = [f(k) for k in range(W, total + 1)]
    assert all(a >= b for a, b in zip(seq, seq[1:]))               # annealing never rises
    # quarter point of the cosine: lr_end + (lr_start - lr_end) (1 + cos(pi/4)) / 2
    assert f(W + 25) == pytest.approx(lr1 + (lr0 - lr1) * (1 + math.sqrt(0.5)) / 2)


def test_loss_weight_pins():
    ws, we = (0.1, 1.0, 0.05), (1.0, 0.5, 0.1)
    assert T.loss_weights(2e-3, 2e-3, ws, we) == pytest.approx(ws)       # x = 1 -> start weights
    assert T.loss_weights(0.0, 2e-3, ws, we) == pytest.approx(we)        # x = 0 -> end weights
    mid = T.loss_weights(1e-3, 2e-3, ws, we)
    assert mid == pytest.approx(tuple((a + b) / 2 for a, b in zip(ws, we)))
    # the printed form takes the learning rate itself as the factor
    assert T.loss_weights(0.25, 1e-3, ws, we, "lr") == pytest.approx(
        tuple(0.25 * a + 0.75 * b for a, b in zip(ws, we)))
    with pytest.raises(ValueError):
        T.loss_weights(1e-3, 1e-3, ws, we, "other")


# --- Adam (Section 3.3.1) ----------------------------------------------------------------
def test_oracle_adam_first_step_and_constant_gradient():
    rng = np.random.default_rng(5)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    g[0] = 0.0
    lr, eps = 1e-3, 1e-8
    # the bias corrections make the first step lr * g / (|g| + eps) exactly
    th1, m, v = O.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr)
    assert np.allclose(theta - th1, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    assert th1[0] == theta[0]
    # a constant gradient keeps mhat = g and vhat = g^2 at every step
    th = th1
    for t in range(2, 40):
        th, m, v = O.adam_step(th, g, m, v, t, lr)
    assert np.allclose(theta - th, 39 * lr * g / (np.abs(g) + eps), rtol=1e-10, atol=1e-15)


def test_oracle_adam_moments():
    rng = np.random.default_rng(6)
    g1, g2 = rng.normal(size=8), rng.normal(size=8)
    _, m, v = O.adam_step(np.zeros(8), g1, np.zeros(8), np.zeros(8), 1, 1e-3)
    _, m, v = O.adam_step(np.zeros(8), g2, m, v, 2, 1e-3)
    assert np.allclose(m, 0.9 * 0.1 * g1 + 0.1 * g2)
    assert np.allclose(v, 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2)


# --- device ------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2607_06969_gb300 import build as B
    B.build()
    from paper_2607_06969_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.gpu
def test_adam_kernel_matches_oracle(nb):
    import torch
    h = I.HYPER_SMALL
    th0 = I.init_params(h).astype(np.float32)
    model = nb.Model(h, th0)
    P = th0.size
    rng = np.random.default_rng(7)
    m1 = torch.zeros(P, dtype=torch.float32, device="cuda")
    m2 = torch.zeros_like(m1)
    th, m, v = th0.astype(np.float64), np.zeros(P), np.zeros(P)
    mabs = np.zeros(P)           # the same average of |g|: the scale of m's rounding
    for t in range(1, 6):
        g = (rng.normal(size=P) * 10.0 ** rng.uniform(-4, 1, size=P)).astype(np.float32)
        lr = 1e-3 * t
        nb.adam_step(model, torch.tensor(g, device="cuda"), m1, m2, t, lr)
        th, m, v = O.adam_step(th, g.astype(np.float64), m, v, t, lr)
        mabs = 0.9 * mabs + 0.1 * np.abs(g)
        got = model.get_params().cpu().numpy().astype(np.float64)
        # FP32 arithmetic on each side of the update: the parameter moves by at
        # most lr per step, so its error stays within a few ulp of |theta|
        assert np.abs(got - th).max() <= 4e-7 * max(1.0, np.abs(th).max()), t
        # m mixes gradients of both signs: its FP32 rounding scales with the
        # average of |g|, not with |m|.  beta2 = 0.999 is held in FP32
        # (0.99900001287...), so 1 - beta2 and the second moment (no
        # cancellation) carry a relative error of 1.3e-5.
        assert np.all(np.abs(m1.cpu().numpy() - m) <= 2e-6 * mabs + 1e-30)
        assert np.allclose(m2.cpu().numpy(), v, rtol=3e-5, atol=1e-30)


@pytest.mark.gpu
def test_adam_argument_errors(nb):
    import torch
    h = I.HYPER_SMALL
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    z = torch.zeros(model.n_params, dtype=torch.float32, device="cuda")
    for kw in (dict(t=0, lr=1e-3), dict(t=1, lr=-1.0), dict(t=1, lr=1e-3, beta1=1.0),
               dict(t=1, lr=1e-3, eps=0.0)):
        with pytest.raises(nb.NepError) as err:
            nb.adam_step(model, z, z.clone(), z.clone(), **kw)
        assert err.value.status == nb.NEP_ERR_ARG


@pytest.mark.gpu
def test_fit_student_to_teacher(nb):
    """Teacher labels from the FP64 oracle (seed-2 weights); the student
    (seed-1 weights) follows the training protocol and its loss, at fixed
    weights, falls well below the start."""
    h = I.HYPER_SMALL
    s = I.packing_batch([24, 40, 57, 33], tag=93)
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    teacher = I.init_params(h, seed=I.SEED_TEACHER).astype(np.float32).astype(np.float64)
    lab = O.energy_forces_virial(h, teacher, p32.astype(np.float64), s.types,
                                 s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)
    model = nb.Model(h, I.init_params(h).astype(np.float32))
    batch = T.make_batch(model, s, lab["Etot"], lab["F"], lab["V"].reshape(-1, 9))
    w = (1.0, 1.0, 0.1)
    loss0 = float(nb.param_grad(model, batch.dsys, batch.nl, batch.ws, batch.e_lbl, batch.f_lbl,
                                batch.v_lbl, w)[1].item())
    cfg = T.TrainConfig(lr_start=3e-3, lr_end=3e-5, epochs=150)
    tr = T.Trainer(model, [batch], cfg)
    for _ in range(cfg.epochs):
        tr.step(batch)
    loss1 = float(nb.param_grad(model, batch.dsys, batch.nl, batch.ws, batch.e_lbl, batch.f_lbl,
                                batch.v_lbl, w)[1].item())
    assert loss1 < 0.3 * loss0, (loss0, loss1)
    # the recorded learning rates follow the schedule (warm-up of one step here)
    lrs = [r["lr"] for r in cfg.history]
    assert lrs[0] == pytest.approx(3e-3 * 1e-4)
    assert lrs[1] == pytest.approx(3e-3)
    assert lrs[-1] == pytest.approx(T.lr_at(149, 3e-3, 3e-5, 1, 150))


@pytest.mark.gpu
def test_checkpoint_resume_is_bit_identical(nb, tmp_path):
    """20 steps straight, or 10 steps, a checkpoint on disk, a fresh model and
    trainer restored from it, and 10 more steps: the same parameters."""
    h = I.HYPER_SMALL
    s = I.packing_batch([24, 40, 33], tag=97)
    p32 = s.pos32()
    pairs = O.neighbor_pairs(p32, s.box, s.atom_off, h.rc_rad)
    teacher = I.init_params(h, seed=I.SEED_TEACHER).astype(np.float32).astype(np.float64)
    lab = O.energy_forces_virial(h, teacher, p32.astype(np.float64), s.types,
                                 s.box.astype(np.float32).astype(np.float64), s.atom_off, pairs)
    th = I.init_params(h).astype(np.float32)

    def trainer():
        model = nb.Model(h, th)
        batch = T.make_batch(model, s, lab["Etot"], lab["F"], lab["V"].reshape(-1, 9))
        return T.Trainer(model, [batch], T.TrainConfig(lr_start=3e-3, lr_end=3e-5, epochs=20)), batch

    a, ba = trainer()
    for _ in range(20):
        a.step(ba)
    b, bb = trainer()
    for _ in range(10):
        b.step(bb)
    path = str(tmp_path / "ckpt.npz")
    b.save(path)
    c, bc = trainer()
    c.load(path)
    for _ in range(10):
        c.step(bc)
    assert np.array_equal(a.model.get_params().cpu().numpy(), c.model.get_params().cpu().numpy())
    assert c.t == 20

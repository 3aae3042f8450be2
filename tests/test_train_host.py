"""Host logic of the training loop (train.Trainer) on the CPU, with the
library calls replaced by a recording stand-in: the learning rate and loss
weights of every step, the Adam step counter, the place of the all-reduce
hook, and the checkpoint round trip."""
import numpy as np
import pytest
import torch

from paper_2607_06969_gb300 import train as T


class FakeModel:
    def __init__(self, P=6):
        self.n_params = P
        self.params = torch.arange(P, dtype=torch.float32)

    def get_params(self):
        return self.params.clone()

    def set_params(self, p):
        self.params = p.clone()


class FakeLib:
    """Stands in for the binding: a gradient of ones, the loss equal to the
    sum of the loss weights, and an update theta -= lr grad."""

    def __init__(self):
        self.calls = []

    def param_grad(self, model, dsys, nl, ws, e, f, v, w, mode, grad=None, loss=None, stream=None):
        self.calls.append(("grad", tuple(w), mode))
        grad.fill_(1.0)
        loss.fill_(float(sum(w)))
        return grad, loss

    def adam_step(self, model, grad, m1, m2, t, lr, beta1, beta2, eps, stream=None):
        self.calls.append(("adam", t, lr, beta1, beta2, eps))
        model.params -= lr * grad


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(T, "nb", lib)
    return lib


def batch(k):
    return T.Batch(dsys=k, nl=None, ws=None, e_lbl=None, f_lbl=None, v_lbl=None)


def test_schedule_weights_and_counter(fake):
    cfg = T.TrainConfig(lr_start=1e-3, lr_end=1e-5, epochs=4)
    tr = T.Trainer(FakeModel(), [batch(0), batch(1), batch(2)], cfg, device="cpu")
    assert tr.warmup == 3 and tr.total == 12
    for _ in range(cfg.epochs):
        tr.epoch()
    adam = [c for c in fake.calls if c[0] == "adam"]
    grads = [c for c in fake.calls if c[0] == "grad"]
    assert [c[1] for c in adam] == list(range(1, 13))            # t = 1, 2, ...
    for k, (a, g) in enumerate(zip(adam, grads)):
        lr = T.lr_at(k, 1e-3, 1e-5, 3, 12)
        assert a[2] == pytest.approx(lr)
        assert g[1] == pytest.approx(T.loss_weights(lr, 1e-3, cfg.w_start, cfg.w_end))
        assert a[3:] == (cfg.beta1, cfg.beta2, cfg.eps)
    assert [h["step"] for h in cfg.history] == list(range(1, 13))
    assert cfg.history[-1]["loss"] == pytest.approx(sum(cfg.history[-1]["w"]))


def test_allreduce_runs_between_gradient_and_update(fake):
    order = []
    tr = T.Trainer(FakeModel(), [batch(0)], T.TrainConfig(epochs=2), device="cpu",
                   allreduce=lambda g, l: order.append(("allreduce", float(g[0]), len(fake.calls))))
    tr.step(tr.batches[0])
    # one gradient call before the hook, the Adam call after it
    assert order == [("allreduce", 1.0, 1)] and fake.calls[1][0] == "adam"


def test_checkpoint_round_trip(fake, tmp_path):
    cfg = T.TrainConfig(epochs=5)
    a = T.Trainer(FakeModel(), [batch(0), batch(1)], cfg, device="cpu")
    for _ in range(3):
        a.step(a.batches[0])
    a.m1 += 0.5
    a.m2 += 0.25
    path = str(tmp_path / "ck.npz")
    a.save(path)
    b = T.Trainer(FakeModel(), [batch(0), batch(1)], T.TrainConfig(epochs=5), device="cpu")
    b.load(path)
    assert b.t == 3 and (b.total, b.warmup) == (a.total, a.warmup)
    assert torch.equal(b.model.get_params(), a.model.get_params())
    assert torch.equal(b.m1, a.m1) and torch.equal(b.m2, a.m2)
    with pytest.raises(ValueError):
        T.Trainer(FakeModel(P=7), [batch(0)], device="cpu").load(path)


def test_table2_preset_runs_the_schedule(fake):
    cfg = T.TrainConfig.table2(epochs=3)
    tr = T.Trainer(FakeModel(), [batch(0)], cfg, device="cpu")
    for _ in range(3):
        tr.step(tr.batches[0])
    lrs = [h["lr"] for h in cfg.history]
    assert lrs[0] == pytest.approx(1e-3 * 1e-4) and lrs[1] == pytest.approx(1e-3)
    assert np.allclose(cfg.history[1]["w"], cfg.w_start)         # lr = lr_start: the start weights

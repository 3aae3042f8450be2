"""Training loop around nep_param_grad (Section 3.3): Adam on the device, a
linear warm-up followed by cosine annealing of the learning rate, and loss
weights interpolated by the learning rate.

Every step runs in libnep kernels (nep_param_grad, then nep_adam_step on the
model's own parameters); this module only schedules the scalars.

Learning rate (Section 3.3.2), stepped once per optimiser step:
  warm-up, steps 0 .. W-1 (W = one epoch):
      lr = lr_start * (f0 + (1 - f0) * step / W),   f0 = 1e-4
  then cosine annealing over the remaining T = total - W steps:
      lr = lr_end + (lr_start - lr_end) * (1 + cos(pi * k / T)) / 2,  k = step - W

Loss weights (Section 3.3.3), per component c in (E, F, V):
      w_c = w_c_start * x + w_c_end * (1 - x)
where the paper writes x = lr (the learning rate itself).  With learning
rates far below 1 that leaves w_c at w_c_end throughout, while the paper's
weight curves (Figs. 7b, 9b) move over the whole run; the reading used by
default is x = lr / lr_start, which runs from ~1 after the warm-up to
lr_end / lr_start at the end.  `weight_factor="lr"` selects the printed form.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import binding as nb


def lr_at(step: int, lr_start: float, lr_end: float, warmup_steps: int, total_steps: int,
          start_factor: float = 1e-4) -> float:
    """Learning rate of optimiser step `step` (0-based)."""
    if warmup_steps > 0 and step < warmup_steps:
        return lr_start * (start_factor + (1.0 - start_factor) * step / warmup_steps)
    T = max(1, total_steps - warmup_steps)
    k = min(step - warmup_steps, T)
    return lr_end + (lr_start - lr_end) * (1.0 + math.cos(math.pi * k / T)) / 2.0


def loss_weights(lr: float, lr_start: float, w_start, w_end, weight_factor: str = "normalised"):
    """(wE, wF, wV) at learning rate lr."""
    if weight_factor == "normalised":
        x = lr / lr_start
    elif weight_factor == "lr":
        x = lr
    else:
        raise ValueError(weight_factor)
    return tuple(float(a * x + b * (1.0 - x)) for a, b in zip(w_start, w_end))


@dataclass
class Batch:
    """One training batch on the device: configurations, their list and the
    labels (E [B] f64, F [3][N] f32, V [B][9] f64)."""
    dsys: nb.DeviceSystem
    nl: nb.NeighborList
    ws: nb.Workspace
    e_lbl: object
    f_lbl: object
    v_lbl: object


@dataclass
class TrainConfig:
    lr_start: float = 1e-3
    lr_end: float = 1e-5
    epochs: int = 10
    w_start: tuple = (0.1, 1.0, 0.05)     # force-heavy early, as in Figs. 7b and 9b
    w_end: tuple = (1.0, 0.5, 0.1)
    weight_factor: str = "normalised"
    loss_mode: int = 0
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    history: list = field(default_factory=list)

    @classmethod
    def table2(cls, **kw) -> "TrainConfig":
        """The training settings of Table 2: lr 1e-3 -> 1e-6 over 200 epochs,
        loss weights (E, F, V) from (0.1, 10, 0.1) to (2, 1, 1).  The table
        prints w_v^end twice; the first of the two rows is read as w_f^end."""
        base = dict(lr_start=1e-3, lr_end=1e-6, epochs=200, w_start=(0.1, 10.0, 0.1), w_end=(2.0, 1.0, 1.0))
        base.update(kw)
        return cls(**base)


class Trainer:
    """Adam over a fixed list of batches, one optimiser step per batch."""

    def __init__(self, model: nb.Model, batches, cfg: TrainConfig | None = None, allreduce=None,
                 device: str = "cuda"):
        """allreduce(grad, loss), if given, combines the ranks' gradients and
        losses in place between nep_param_grad and the Adam step (data
        parallelism, see dp.allreduce_mean)."""
        import torch
        self.allreduce = allreduce
        self.model = model
        self.batches = list(batches)
        self.cfg = cfg or TrainConfig()
        self.device = device
        P = model.n_params
        self.m1 = torch.zeros(P, dtype=torch.float32, device=device)
        self.m2 = torch.zeros(P, dtype=torch.float32, device=device)
        self.grad = torch.empty(P, dtype=torch.float32, device=device)
        self.loss = torch.empty(1, dtype=torch.float64, device=device)
        self.t = 0
        self.total = self.cfg.epochs * len(self.batches)
        self.warmup = len(self.batches)           # one epoch

    def step(self, batch: Batch, stream=None) -> float:
        """One optimiser step on `batch`; returns the loss before the update
        (read back to the host, so this synchronises)."""
        c = self.cfg
        lr = lr_at(self.t, c.lr_start, c.lr_end, self.warmup, self.total)
        w = loss_weights(lr, c.lr_start, c.w_start, c.w_end, c.weight_factor)
        nb.param_grad(self.model, batch.dsys, batch.nl, batch.ws, batch.e_lbl, batch.f_lbl, batch.v_lbl,
                      w, c.loss_mode, grad=self.grad, loss=self.loss, stream=stream)
        if self.allreduce is not None:
            self.allreduce(self.grad, self.loss)
        self.t += 1
        nb.adam_step(self.model, self.grad, self.m1, self.m2, self.t, lr, c.beta1, c.beta2, c.eps,
                     stream=stream)
        loss = float(self.loss.item())
        c.history.append({"step": self.t, "lr": lr, "w": w, "loss": loss})
        return loss

    def epoch(self, stream=None) -> float:
        return float(np.mean([self.step(b, stream) for b in self.batches]))

    # --- checkpoint / resume --------------------------------------------------
    def state_dict(self) -> dict:
        """Everything a resumed run needs: parameters, Adam moments, the step
        counter (which also fixes the learning rate and loss weights)."""
        return {"params": self.model.get_params().cpu().numpy().copy(),
                "m1": self.m1.cpu().numpy().copy(), "m2": self.m2.cpu().numpy().copy(),
                "t": self.t, "total": self.total, "warmup": self.warmup}

    def load_state_dict(self, st: dict) -> None:
        import torch
        if st["params"].size != self.model.n_params:
            raise ValueError("checkpoint has %d parameters, the model %d" % (st["params"].size,
                                                                               self.model.n_params))
        self.model.set_params(torch.tensor(np.asarray(st["params"], np.float32), device=self.device))
        self.m1.copy_(torch.tensor(np.asarray(st["m1"], np.float32)))
        self.m2.copy_(torch.tensor(np.asarray(st["m2"], np.float32)))
        self.t, self.total, self.warmup = int(st["t"]), int(st["total"]), int(st["warmup"])
        if self.device != "cpu":
            torch.cuda.synchronize()

    def save(self, path: str) -> None:
        np.savez(path, **{k: np.asarray(v) for k, v in self.state_dict().items()})

    def load(self, path: str) -> None:
        with np.load(path) as z:
            self.load_state_dict({k: z[k] for k in z.files})


def make_batch(model: nb.Model, s, e_lbl, f_lbl, v_lbl, cap: int = 112, cap_ang: int = 56) -> Batch:
    """Device batch for the System `s` with host labels (E [B], F [N,3], V [B,9])."""
    import torch
    dsys = nb.DeviceSystem.from_inputs(s)
    nl = nb.NeighborList(s.n_atoms, cap, cap_ang)
    ws = nb.Workspace(model, s.n_atoms, s.n_cfg, cap, cap_ang, train=True)
    nb.neighbors(model, dsys, nl, 0.0, ws)
    if nb.check_list(nl) != nb.NEP_OK:
        raise nb.NepError(nb.check_list(nl), "neighbours", nb.last_error())
    return Batch(dsys, nl, ws,
                 torch.tensor(np.asarray(e_lbl, np.float64), device="cuda"),
                 torch.tensor(np.ascontiguousarray(np.asarray(f_lbl, np.float32).T), device="cuda"),
                 torch.tensor(np.asarray(v_lbl, np.float64).reshape(-1, 9), device="cuda"))

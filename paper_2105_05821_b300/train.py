"""Training the latency predictor (Sec. 2.4) through the library's hand-written
backward kernels.

* `Windows`: a labelled trace resident on the device (records, fetch cycles,
  execution-latency labels, first in-flight instruction of every window,
  (F, E) targets), built from the toy pipeline model's labels.
* `CNNFunction`: a torch.autograd.Function whose forward and backward are
  simnet_train_forward / simnet_train_backward; the parameters are one flat
  FP32 tensor in the canonical blob layout, so any torch optimiser can drive it.
* `LossFunction`: the training loss (squared error of softplus, plus the class
  cross-entropy with the hybrid head) as a torch.autograd.Function over
  simnet_train_loss: the library's loss kernels compute the loss and dz.
* `train`: the library's own fused step (gather, forward, loss, backward, Adam).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import inputs as I
from .simnet import Simnet


@dataclass
class Windows:
    records: torch.Tensor     # int32 [N]
    fetch: torch.Tensor       # int64 [N]
    e_label: torch.Tensor     # uint8 [N]
    ctx_begin: torch.Tensor   # int64 [N]
    labels: torch.Tensor      # uint8 [N, 2]

    @staticmethod
    def from_labels(records: np.ndarray, L: I.Labels, device="cuda") -> "Windows":
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
        return Windows(t(records.view(np.int32)), t(L.fetch), t(L.E), t(L.ctx_begin),
                       t(np.stack([L.F, L.E], 1)))

    def __len__(self) -> int:
        return self.records.numel()


class CNNFunction(torch.autograd.Function):
    """z = CNN(x; w) with w the canonical flat weight tensor (FP32, on the device)."""

    @staticmethod
    def forward(ctx, x, w, sim: Simnet):
        sim.set_weights_device(w.detach().contiguous())
        z = sim.train_forward(x.contiguous())
        ctx.sim = sim
        return z

    @staticmethod
    def backward(ctx, dz):
        g = ctx.sim.train_backward(dz.contiguous().float())
        return None, g, None


class LossFunction(torch.autograd.Function):
    """loss = the library's training loss of FC2 outputs z [n, n_out] against
    uint8 latency labels [n, 2] (Sec. 2.4; with the hybrid head Sec. 2.3's
    cross-entropy is added).  Forward and backward are simnet_train_loss."""

    @staticmethod
    def forward(ctx, z, labels, sim: Simnet):
        z = z.detach().contiguous().float()
        labels = labels.contiguous()
        loss = torch.empty((), dtype=torch.float32, device=z.device)
        sim.train_loss(z, labels, loss=loss)
        ctx.save_for_backward(z, labels)
        ctx.sim = sim
        return loss

    @staticmethod
    def backward(ctx, g):
        z, labels = ctx.saved_tensors
        dz = torch.empty_like(z)
        gs = g.detach().reshape(1).contiguous().float()
        ctx.sim.train_loss(z, labels, grad_scale=gs, dz=dz)
        return dz, None, None


def train(sim: Simnet, w: Windows, steps: int, batch: int, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Fused library training steps on random windows; returns the loss per step."""
    g = torch.Generator(device=w.records.device)
    g.manual_seed(seed)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, len(w), (batch,), device=w.records.device, generator=g)
        losses.append(sim.train_step(w, idx, lr))
        if log_every and s % log_every == 0:
            print(f"step {s}: loss {losses[-1]:.4f}")
    return losses

"""Training the latency predictor (Sec. 2.4) through the library's hand-written
backward kernels.

* `Windows`: a labelled trace resident on the device (records, fetch cycles,
  execution-latency labels, first in-flight instruction of every window,
  (F, E) targets), built from the toy pipeline model's labels.
* `CNNFunction`: a torch.autograd.Function whose forward and backward are
  simnet_train_forward / simnet_train_backward; the parameters are one flat
  FP32 tensor in the canonical blob layout, so any torch optimiser can drive it.
* `train`: the library's own fused step (gather, forward, MSE, backward, Adam).
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


def mse_softplus(z: torch.Tensor, labels: torch.Tensor) -> torch.Tensor:
    """Mean over all outputs of (softplus(z) - clamp(label, 0, 255))^2."""
    return (torch.nn.functional.softplus(z) - labels.float().clamp(0, 255)).pow(2).mean()


def hybrid_loss(z: torch.Tensor, labels: torch.Tensor) -> torch.Tensor:
    """Hybrid head (Sec. 2.3) loss on z [n, 22]: mean over the 2n latencies of the
    cross-entropy of the ten class logits against class min(label, 9) plus the
    squared error of softplus(regression output) against the label."""
    y = labels.float().clamp(0, 255)
    total = z.new_zeros(())
    for t in range(2):
        cls = y[:, t].clamp(max=9).long()
        ce = torch.nn.functional.cross_entropy(z[:, 11 * t:11 * t + 10], cls, reduction="sum")
        se = (torch.nn.functional.softplus(z[:, 11 * t + 10]) - y[:, t]).pow(2).sum()
        total = total + ce + se
    return total / (2 * z.shape[0])


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

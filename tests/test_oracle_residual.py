"""Pins of the oracle's residual-block CNN (the RB models of Sec. 2.3), without
a GPU: the forward pass against a PyTorch float64 model written with
torch.nn.functional (k=2 / stride-2 conv1d + ReLU, pointwise conv1d, bias-free
k=2 / stride-2 projection shortcut, add, ReLU), and two reductions that make
the block a plain layer."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import oracle
from paper_2105_05821_b300 import inputs as I


def rb(arch: I.Arch, head: str = "regression") -> I.Arch:
    return I.Arch(arch.window, arch.n_conv, arch.channels, arch.hidden, head, block="residual")


def torch_rb_forward(arch: I.Arch, blob: np.ndarray, x: np.ndarray):
    ws = {k: torch.tensor(v, dtype=torch.float64) for k, v in I.unflatten_weights(arch, blob)}
    h = torch.tensor(x, dtype=torch.float64).permute(0, 2, 1)      # [n, 50, W]
    for k in range(1, arch.n_conv + 1):
        a = torch.relu(Fn.conv1d(h, ws[f"rb{k}.conv.weight"], ws[f"rb{k}.conv.bias"], stride=2))
        s = Fn.conv1d(h, ws[f"rb{k}.proj.weight"], None, stride=2)
        h = torch.relu(Fn.conv1d(a, ws[f"rb{k}.pw.weight"], ws[f"rb{k}.pw.bias"]) + s)
    h = h.reshape(h.shape[0], -1)
    h = torch.relu(Fn.linear(h, ws["fc1.weight"], ws["fc1.bias"]))
    return Fn.linear(h, ws["fc2.weight"], ws["fc2.bias"]).numpy()


@pytest.mark.parametrize("arch", [rb(I.Arch(32, 3, 16, 24)), rb(I.Arch(16, 2, 8, 12), "hybrid"),
                                  rb(I.Arch(8, 1, 5, 3)), rb(I.Arch(128, 7, 8, 16))])
def test_residual_forward_matches_torch_float64(arch):
    cfg = oracle.Config.of(arch)
    assert cfg.residual and oracle.blob_size(cfg) == arch.n_params()
    blob = I.flatten_weights(I.he_weights(arch, 4, bias_std=0.3))
    x = I.random_windows(20, arch, 8)
    np.testing.assert_allclose(oracle.cnn_forward(cfg, blob, x), torch_rb_forward(arch, blob, x),
                               rtol=1e-12, atol=1e-12)


def to_plain(arch: I.Arch, blob: np.ndarray, keep: str) -> np.ndarray:
    """The plain-CNN blob whose layer k is the residual block's conv (keep =
    "conv") or its projection with the conv's bias (keep = "proj")."""
    ws = dict(I.unflatten_weights(arch, blob))
    plain = I.Arch(arch.window, arch.n_conv, arch.channels, arch.hidden, arch.head)
    out = []
    for name, _ in plain.shapes():
        if name.startswith("conv"):
            k, kind = name[4:].split(".")
            src = f"rb{k}.{keep}.weight" if kind == "weight" else f"rb{k}.conv.bias"
            out.append(ws[src])
        else:
            out.append(ws[name])
    return np.concatenate([np.asarray(a).ravel() for a in out])


def test_block_reduces_to_its_conv_without_shortcut():
    """proj = 0, pw = identity, pw bias = 0: y = ReLU(ReLU(conv x)) = ReLU(conv x)."""
    arch = rb(I.Arch(32, 3, 16, 24))
    ws = I.he_weights(arch, 6, bias_std=0.2)
    ws = [(n, np.zeros_like(a) if n.endswith("proj.weight") or n.endswith("pw.bias") else
           (np.eye(16)[:, :, None] if n.endswith("pw.weight") else a)) for n, a in ws]
    blob = I.flatten_weights(ws)
    x = I.random_windows(10, arch, 3)
    plain = I.Arch(32, 3, 16, 24)
    np.testing.assert_allclose(oracle.cnn_forward(oracle.Config.of(arch), blob, x),
                               oracle.cnn_forward(oracle.Config.of(plain), to_plain(arch, blob, "conv"), x),
                               rtol=1e-13, atol=1e-13)


def test_block_reduces_to_its_shortcut_without_branch():
    """pw = 0: y = ReLU(pw bias + proj x); with the conv bias copied into the pw
    bias that is a plain layer with the projection's weights."""
    arch = rb(I.Arch(16, 2, 8, 12))
    ws = dict(I.he_weights(arch, 7, bias_std=0.2))
    for k in (1, 2):
        ws[f"rb{k}.pw.weight"] = np.zeros_like(ws[f"rb{k}.pw.weight"])
        ws[f"rb{k}.pw.bias"] = ws[f"rb{k}.conv.bias"].copy()
    blob = I.flatten_weights([(n, ws[n]) for n, _ in arch.shapes()])
    x = I.random_windows(10, arch, 5)
    plain = I.Arch(16, 2, 8, 12)
    np.testing.assert_allclose(oracle.cnn_forward(oracle.Config.of(arch), blob, x),
                               oracle.cnn_forward(oracle.Config.of(plain), to_plain(arch, blob, "proj"), x),
                               rtol=1e-13, atol=1e-13)


def test_training_loss_refuses_residual_blocks():
    arch = rb(I.Arch(16, 2, 8, 12))
    with pytest.raises(ValueError):
        oracle.loss_grad(oracle.Config.of(arch), np.zeros(arch.n_params()), I.random_windows(2, arch, 1),
                         np.zeros((2, 2)))

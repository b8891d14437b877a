"""Pins of the oracle's CNN, loss gradient and Adam step (no GPU).

The oracle's plain loops are checked against independent library routines
(PyTorch float64 conv1d / linear / autograd / Adam) and against central finite
differences (Sec. 2.3 architecture, Sec. 2.4 training).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import oracle
from paper_2105_05821_b300 import inputs as I


def torch_forward(arch: I.Arch, blob: np.ndarray, x: np.ndarray, grad=False):
    ws = {k: torch.tensor(v, dtype=torch.float64, requires_grad=grad)
          for k, v in I.unflatten_weights(arch, blob)}
    h = torch.tensor(x, dtype=torch.float64).permute(0, 2, 1)      # [n, 50, W]
    for k in range(arch.n_conv):
        h = torch.relu(Fn.conv1d(h, ws[f"conv{k + 1}.weight"], ws[f"conv{k + 1}.bias"], stride=2))
    h = h.reshape(h.shape[0], -1)                                   # PyTorch flatten: c*L + l
    h = torch.relu(Fn.linear(h, ws["fc1.weight"], ws["fc1.bias"]))
    z = Fn.linear(h, ws["fc2.weight"], ws["fc2.bias"])
    return z, ws


@pytest.mark.parametrize("arch", [I.Arch(32, 2, 64, 256), I.Arch(16, 3, 8, 12),
                                  I.Arch(8, 1, 5, 3), I.Arch(128, 5, 16, 32)])
def test_cnn_matches_torch_float64(arch):
    cfg = oracle.Config.of(arch)
    blob = I.flatten_weights(I.he_weights(arch, 4, bias_std=0.3))
    x = I.random_windows(24, arch, 8)
    z = oracle.cnn_forward(cfg, blob, x)
    zt, _ = torch_forward(arch, blob, x)
    np.testing.assert_allclose(z, zt.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_softplus_closed_form():
    z = np.array([-30.0, -1.0, 0.0, 1.0, 19.9, 20.0, 20.1, 50.0])
    sp = oracle.softplus(z)
    assert sp[2] == pytest.approx(np.log(2.0), abs=1e-15)
    np.testing.assert_allclose(sp[1] - oracle.softplus(-z)[1], z[1], atol=1e-15)  # sp(x)-sp(-x)=x
    assert sp[6] == 20.1 and sp[7] == 50.0                                      # identity above 20


def _small():
    arch = I.Arch(8, 2, 4, 6)
    cfg = oracle.Config.of(arch)
    blob = I.flatten_weights(I.he_weights(arch, 21, bias_std=0.2))
    x = I.random_windows(5, arch, 22)
    y = np.random.default_rng(23).integers(0, 12, (5, 2)).astype(np.float64)
    return arch, cfg, blob, x, y


def test_grad_matches_torch_autograd():
    arch, cfg, blob, x, y = _small()
    loss, g = oracle.loss_grad(cfg, blob, x, y)
    z, ws = torch_forward(arch, blob, x, grad=True)
    lt = ((Fn.softplus(z) - torch.tensor(y).clamp(0, 255)) ** 2).mean()
    lt.backward()
    gt = np.concatenate([ws[k].grad.numpy().ravel() for k, _ in arch.shapes()])
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    np.testing.assert_allclose(g, gt, rtol=1e-10, atol=1e-13)


def test_grad_matches_finite_differences():
    """Central differences, h = 1e-6, on every parameter of a small CNN."""
    arch, cfg, blob, x, y = _small()
    _, g = oracle.loss_grad(cfg, blob, x, y)
    h = 1e-6
    fd = np.zeros_like(blob)
    for i in range(len(blob)):
        bp, bm = blob.copy(), blob.copy()
        bp[i] += h
        bm[i] -= h
        fd[i] = (oracle.loss_grad(cfg, bp, x, y)[0] - oracle.loss_grad(cfg, bm, x, y)[0]) / (2 * h)
    err = np.abs(fd - g) / (np.abs(g) + 1e-6)
    # a coordinate whose +-h flips a ReLU may differ; there should be (almost) none
    assert np.mean(err < 1e-5) > 0.99, np.sort(err)[-5:]


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        oracle.adam(theta, m, v, g.copy(), t=t)
        p.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_window_features_hand():
    """Training windows: row 0 = instruction i; rows 1.. = i-1, i-2, ... down to
    the first instruction still in flight; residence against fetch[i-1]."""
    insts = [[3, 1, 2, 5, 1, 0, 0, 1, 0], [7, 5, 9, 6, 0, 1, 0, 1, 0], [31, 6, 5, 0, 0, 0, 1, 0, 1]]
    recs = I.pack_records(*np.array(insts).T)
    fetch = np.array([0, 2, 5], np.int64)
    e_lab = np.array([7, 3, 1], np.uint8)
    ctx_begin = np.array([0, 0, 1], np.int64)
    cfg = oracle.Config(window=4, n_conv=1, channels=2, hidden=2)
    X = oracle.window_features(cfg, recs, fetch, e_lab, ctx_begin, [2, 1, 0])
    # window of instruction 2: context is instruction 1 only (instruction 0 has committed)
    assert X[0, 0, 31] == 1 and X[0, 0, 37] == 1 and X[0, 0, 41] == 1
    assert X[0, 1, 7] == 1 and X[0, 1, 42] == 0.0 and X[0, 1, 43] == 3 / 64 and X[0, 1, 45] == 1
    assert not X[0, 2:].any()
    # window of instruction 1: instruction 0 with residence fetch[0]-fetch[0] = 0, E = 7
    assert X[1, 1, 3] == 1 and X[1, 1, 42] == 0.0 and X[1, 1, 43] == 7 / 64
    assert X[1, 1, 45] == 1 and X[1, 1, 46] == 0   # dst of 0 (r5) is src0 of 1
    assert X[1, 1, 48] == 1                        # 0 is a load, 1 a store, both at L2
    assert not X[2, 1:].any()

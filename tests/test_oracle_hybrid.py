"""Pins of the oracle's hybrid head (Sec. 2.3: per latency 10 class logits for
0..8 cycles and "more than 8", plus a regression output used for the last
class) and of its training loss (cross-entropy + squared error), without a GPU.

Independent references: PyTorch float64 linear / cross_entropy / autograd,
central finite differences, and whole simulations whose FC2 is reduced to its
bias (w2 = 0) so that every decision is known in advance and the cycle count
follows from the stub-predictor path.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import oracle
from paper_2105_05821_b300 import inputs as I

from test_oracle_cnn import torch_forward


def hybrid(arch: I.Arch) -> I.Arch:
    return I.Arch(arch.window, arch.n_conv, arch.channels, arch.hidden, "hybrid")


@pytest.mark.parametrize("arch", [hybrid(I.Arch(32, 2, 64, 256)), hybrid(I.Arch(16, 3, 8, 12))])
def test_hybrid_forward_matches_torch_float64(arch):
    cfg = oracle.Config.of(arch)
    assert cfg.hybrid and cfg.n_out == 22 and oracle.blob_size(cfg) == arch.n_params()
    blob = I.flatten_weights(I.he_weights(arch, 5, bias_std=0.3))
    x = I.random_windows(16, arch, 9)
    z = oracle.cnn_forward(cfg, blob, x)
    zt, _ = torch_forward(arch, blob, x)
    assert z.shape == (16, 22)
    np.testing.assert_allclose(z, zt.detach().numpy(), rtol=1e-12, atol=1e-12)


def _small():
    arch = hybrid(I.Arch(8, 2, 4, 6))
    cfg = oracle.Config.of(arch)
    blob = I.flatten_weights(I.he_weights(arch, 31, bias_std=0.2))
    x = I.random_windows(7, arch, 32)
    # labels up to 15: classes 0..8 and "more than 8", with an O(1) loss (larger labels make
    # the squared error so large that central differences lose their accuracy)
    y = np.array([[0, 3], [1, 9], [8, 14], [2, 0], [12, 5], [0, 15], [5, 8]], dtype=np.float64)
    return arch, cfg, blob, x, y


def torch_hybrid_loss(z, y):
    """Mean over the 2n latencies of CE(class logits, min(y, 9)) + (softplus(value) - y)^2."""
    yt = torch.tensor(y).clamp(0, 255)
    terms = []
    for t in range(2):
        cls = torch.clamp(yt[:, t], max=9).long()
        ce = Fn.cross_entropy(z[:, 11 * t:11 * t + 10], cls, reduction="none")
        se = (Fn.softplus(z[:, 11 * t + 10]) - yt[:, t]) ** 2
        terms.append(ce + se)
    return torch.stack(terms, 1).mean()


def test_hybrid_loss_and_grad_match_torch_autograd():
    arch, cfg, blob, x, y = _small()
    loss, g = oracle.loss_grad(cfg, blob, x, y)
    z, ws = torch_forward(arch, blob, x, grad=True)
    lt = torch_hybrid_loss(z, y)
    lt.backward()
    gt = np.concatenate([ws[k].grad.numpy().ravel() for k, _ in arch.shapes()])
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    np.testing.assert_allclose(g, gt, rtol=1e-10, atol=1e-13)


def test_hybrid_grad_matches_finite_differences():
    arch, cfg, blob, x, y = _small()
    _, g = oracle.loss_grad(cfg, blob, x, y)
    h = 1e-6
    err = []
    for i in range(len(blob)):
        bp, bm = blob.copy(), blob.copy()
        bp[i] += h
        bm[i] -= h
        fd = (oracle.loss_grad(cfg, bp, x, y)[0] - oracle.loss_grad(cfg, bm, x, y)[0]) / (2 * h)
        err.append(abs(fd - g[i]) - 1e-5 * abs(g[i]))
    # the loss is O(10) (cross-entropy terms), so a central difference carries ~1e-8 of
    # rounding noise: an absolute bound for small gradients, relative for large ones
    assert np.mean(np.array(err) < 1e-7) > 0.99, np.sort(err)[-5:]


# ---------------------------------------------------------------- decisions through simulation
def bias_only_blob(arch: I.Arch, logits_f, value_f, logits_e, value_e) -> np.ndarray:
    """A hybrid blob whose FC2 weights are zero: every instruction's FC2 outputs
    equal the biases given here."""
    ws = I.he_weights(arch, 3)
    b2 = np.concatenate([logits_f, [value_f], logits_e, [value_e]]).astype(np.float64)
    ws[-2] = ("fc2.weight", np.zeros_like(ws[-2][1]))
    ws[-1] = ("fc2.bias", b2)
    return I.flatten_weights(ws)


def run(arch, blob, trace, replay=None):
    cfg = oracle.Config.of(arch)
    return oracle.simulate(cfg, trace.records, trace.offsets, blob, replay=replay, logs=True)


@pytest.mark.parametrize("fetch_class,exec_value,expect_f,expect_e", [
    (3, 2.0, 3, 2),          # class 3 wins for fetch; execution falls to the regression output
    (0, 12.0, 0, 12),        # F = 0: no retire budget until the drain
    (8, 0.3, 8, 1),          # the last direct class; softplus(0.3) = 0.854 -> 1
])
def test_hybrid_decisions_drive_the_simulation(fetch_class, exec_value, expect_f, expect_e):
    arch = hybrid(I.Arch(16, 2, 4, 8))
    lf = np.zeros(10)
    lf[fetch_class] = 2.0
    le = np.zeros(10)
    le[9] = 5.0                                   # "more than 8" wins for the execution latency
    blob = bias_only_blob(arch, lf, -50.0, le, exec_value)
    trace = I.small_trace([40, 7, 1], seed=3)
    r = run(arch, blob, trace)
    assert (r.lat[:, 0] == expect_f).all() and (r.lat[:, 1] == expect_e).all()
    np.testing.assert_allclose(r.pre[:, 1], np.log1p(np.exp(exec_value)), rtol=1e-15)
    # the same constant latencies through the stub-predictor path give the same cycles
    stub = np.tile(np.array([expect_f, expect_e], np.uint8), (trace.n_instructions, 1))
    s = oracle.simulate(oracle.Config.of(arch), trace.records, trace.offsets, replay=stub)
    np.testing.assert_array_equal(r.cycles, s.cycles)


def test_hybrid_largest_logit_lowest_class_on_exact_ties():
    """The class with the largest probability (Sec. 2.3) is the largest logit,
    compared in FP64: an exact tie takes the lower class, a gap of 1e-12 is
    enough to decide."""
    arch = hybrid(I.Arch(16, 2, 4, 8))
    trace = I.small_trace([5], seed=4)
    lf = np.zeros(10)
    lf[2] = lf[6] = 1.5                           # an exact tie: class 2
    le = np.zeros(10)
    le[4], le[5] = 1.0, 1.0 + 1e-12               # larger in FP64 (equal once rounded to FP32): class 5
    r = run(arch, bias_only_blob(arch, lf, 0.0, le, 0.0), trace)
    assert (r.lat[:, 0] == 2).all() and (r.lat[:, 1] == 5).all()


def test_hybrid_with_class_nine_always_winning_is_the_regression_model():
    """If "more than 8" always wins, the hybrid head predicts exactly what a
    regression head with the same value rows predicts."""
    reg = I.Arch(16, 2, 8, 12)
    hyb = hybrid(reg)
    wr = I.he_weights(reg, 7, bias_std=0.3)
    wh = I.he_weights(hyb, 7, bias_std=0.3)   # same draws up to FC2
    for k in range(len(wr) - 2):
        wh[k] = wr[k]
    w2r, b2r = wr[-2][1], wr[-1][1]
    w2h = np.zeros((22, reg.hidden))
    b2h = np.zeros(22)
    for t in range(2):
        w2h[11 * t + 10] = w2r[t]
        b2h[11 * t + 10] = b2r[t]
        b2h[11 * t + 9] = 100.0                   # class 9 wins every time
    wh[-2] = ("fc2.weight", w2h)
    wh[-1] = ("fc2.bias", b2h)
    trace = I.small_trace([60, 33], seed=8)
    a = run(reg, I.flatten_weights(wr), trace)
    b = run(hyb, I.flatten_weights(wh), trace)
    np.testing.assert_array_equal(a.lat, b.lat)
    np.testing.assert_array_equal(a.cycles, b.cycles)
    np.testing.assert_array_equal(a.pre, b.pre)


def test_head_decision_on_given_outputs():
    """oracle.head on hand-set FC2 outputs: direct classes, the "more than 8"
    class through softplus of the regression output, exact ties, a gap of
    1e-12 decided in FP64, and the regression head's plain rounding."""
    cfg = oracle.Config.of(hybrid(I.Arch(16, 2, 4, 8)))
    z = np.zeros((3, 22))
    z[0, 4] = 1.0                                  # fetch: class 4
    z[0, 11 + 9], z[0, 21] = 2.0, 30.0             # execution: class 9, softplus(30) = 30
    z[1, 0] = z[1, 7] = 0.5                        # exact tie: lowest index
    z[1, 11 + 2], z[1, 11 + 3] = 0.25, 0.25 + 1e-12    # decided in FP64: class 3
    z[2, 9], z[2, 10] = 1.0, -50.0                 # class 9 with a value that rounds to 0
    z[2, 11 + 8] = 3.0
    lat, pre = oracle.head(cfg, z)
    np.testing.assert_array_equal(lat, [[4, 30], [0, 3], [0, 8]])
    np.testing.assert_allclose(pre[:, 1], oracle.softplus(z[:, 21]), rtol=1e-15)
    reg = oracle.Config.of(I.Arch(16, 2, 4, 8))
    lat, pre = oracle.head(reg, np.array([[0.0, 3.4], [-60.0, 300.0]]))
    np.testing.assert_array_equal(lat, [[1, 3], [0, 255]])   # softplus(0) = 0.693 -> 1

"""GPU parity of training (Sec. 2.4): the library's window gather, forward,
hand-written backward, loss and Adam against the FP64 oracle (which is itself
pinned to PyTorch autograd and central finite differences), plus a
training-sanity run on toy-pipeline labels.  FP32 contexts train on the CUDA
cores; BF16 contexts on the tcgen05 tensor cores (BF16 operands, FP32 sums),
whose gradients are held to the BF16 bounds below."""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.train import CNNFunction, LossFunction, Windows, train

from gpu_util import hybrid_loss, latency_error, make_sim, mse_softplus
from tolerances import check

pytestmark = pytest.mark.gpu

ARCH = I.ARCH_SMALL(96)     # the training workload's CNN: W=96, 2xConv64, FC256


@pytest.fixture(scope="module")
def data():
    rec = I.make_records(6000, 33)
    L = I.toy_labels(rec)
    return rec, L, Windows.from_labels(rec, L)


def oracle_windows(rec, L, idx):
    cfg = oracle.Config.of(ARCH)
    return oracle.window_features(cfg, rec, L.fetch, L.E, L.ctx_begin, idx)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_gather_windows_exact(data):
    rec, L, w = data
    idx = np.array([0, 1, 2, 63, 64, 65, 777, 4096, 5999])
    sim, _ = make_sim(ARCH, "fp32", seed=3)
    x = sim.gather_windows(w, torch.from_numpy(idx).cuda()).cpu().numpy()
    np.testing.assert_array_equal(x, oracle_windows(rec, L, idx).astype(np.float32))


# precision -> (loss, relative L2 of the whole gradient, of each parameter tensor)
GRAD_TOL = {"fp32": (1e-4, 1e-4, 1e-3), "bf16": (1e-2, 2e-2, 5e-2)}


@pytest.mark.parametrize("n", [256, 300])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_forward_backward_match_oracle_gradient(data, precision, n):
    """CNNFunction and LossFunction (the library's forward, loss and backward
    kernels behind torch.autograd) against the oracle's FP64 loss and gradient;
    300 windows leave a ragged tail in every GEMM."""
    rec, L, w = data
    idx = np.random.default_rng(5).integers(0, len(rec), n)
    blob = I.workload_weights(I.Workload("t", ARCH, 1, 1, seed=3))
    cfg = oracle.Config.of(ARCH)
    x = oracle_windows(rec, L, idx)
    y = np.stack([L.F[idx], L.E[idx]], 1).astype(np.float64)
    loss_o, g_o = oracle.loss_grad(cfg, blob, x, y)
    sim, _ = make_sim(ARCH, precision, blob=blob)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    wt = torch.from_numpy(blob.astype(np.float32)).cuda().requires_grad_(True)
    z = CNNFunction.apply(xt, wt, sim)
    loss = LossFunction.apply(z, torch.from_numpy(y.astype(np.uint8)).cuda(), sim)
    loss.backward()
    tl, tg, tt = GRAD_TOL[precision]
    zr = oracle.cnn_forward(cfg, blob, x)
    check(latency_error(z.detach().cpu().numpy(), zr), precision, f"training forward, {n} windows")
    assert loss.item() == pytest.approx(loss_o, rel=tl)
    g = wt.grad.cpu().numpy().astype(np.float64)
    assert rel(g, g_o) < tg, rel(g, g_o)
    # per parameter tensor as well (the small ones must not hide in the norm)
    k = 0
    for name, shape in ARCH.shapes():
        m = int(np.prod(shape))
        assert rel(g[k:k + m], g_o[k:k + m]) < tt, (name, rel(g[k:k + m], g_o[k:k + m]))
        k += m


@pytest.mark.parametrize("hybrid", [False, True])
def test_library_loss_matches_torch_statement(hybrid):
    """simnet_train_loss (through LossFunction) against the plain PyTorch
    statement of the same loss, value and gradient, with an incoming gradient
    of 3 (the chain rule's scale)."""
    arch = I.Arch(96, 2, 64, 256, "hybrid" if hybrid else "regression")
    sim, _ = make_sim(arch, "fp32")
    g = torch.Generator(device="cuda").manual_seed(4)
    n = 777
    z = (torch.randn((n, arch.n_out), device="cuda", generator=g) * 4).requires_grad_(True)
    z[:3, :].data.fill_(30.0)                            # above the softplus threshold
    lab = torch.randint(0, 256, (n, 2), device="cuda", generator=g, dtype=torch.int32).to(torch.uint8)
    lab[:50] = torch.randint(0, 10, (50, 2), device="cuda", generator=g, dtype=torch.int32).to(torch.uint8)
    loss = LossFunction.apply(z, lab, sim)
    (3.0 * loss).backward()
    zr = z.detach().double().requires_grad_(True)
    ref = (hybrid_loss if hybrid else mse_softplus)(zr, lab)
    (3.0 * ref).backward()
    assert loss.item() == pytest.approx(ref.item(), rel=1e-5)
    d = (z.grad.double() - zr.grad).abs().max().item()
    assert d <= 1e-6 * (zr.grad.abs().max().item() + 1e-12) + 1e-9, d


def test_gradient_against_finite_differences(data):
    """The GPU gradient on 64 windows against FP64 central differences of the
    oracle's loss, on a sample of coordinates from every parameter tensor."""
    rec, L, w = data
    idx = np.random.default_rng(8).integers(0, len(rec), 64)
    # non-zero biases: with zero conv biases every all-zero input row (short
    # context) sits exactly on a ReLU kink, where a central difference averages
    # the two one-sided slopes and no gradient convention can match it
    blob = I.workload_weights(I.Workload("t", ARCH, 1, 1, seed=4))
    k = 0
    for name, shape in ARCH.shapes():
        n = int(np.prod(shape))
        if name.endswith("bias") and not name.startswith("fc2"):
            blob[k:k + n] = np.random.default_rng(k).normal(0, 0.05, n)
        k += n
    cfg = oracle.Config.of(ARCH)
    x = oracle_windows(rec, L, idx)
    y = np.stack([L.F[idx], L.E[idx]], 1).astype(np.float64)
    sim, _ = make_sim(ARCH, "fp32", blob=blob)
    z = sim.train_forward(torch.from_numpy(x.astype(np.float32)).cuda())
    zz = z.double().cpu().numpy()
    sp = oracle.softplus(zz)
    dz = (sp - y) / len(idx) * np.where(zz > 20, 1.0, 1.0 / (1.0 + np.exp(-zz)))
    g = sim.train_backward(torch.from_numpy(dz.astype(np.float32)).cuda()).double().cpu().numpy()
    rng = np.random.default_rng(9)
    k, coords = 0, []
    for name, shape in ARCH.shapes():
        n = int(np.prod(shape))
        coords += list(k + rng.choice(n, min(n, 4), replace=False))
        k += n
    h = 1e-6
    for i in coords:
        bp, bm = blob.copy(), blob.copy()
        bp[i] += h
        bm[i] -= h
        fd = (oracle.loss_grad(cfg, bp, x, y)[0] - oracle.loss_grad(cfg, bm, x, y)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-3 * abs(fd) + 1e-6, (i, g[i], fd)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_train_step_matches_oracle_adam(data, precision):
    rec, L, w = data
    idx = np.random.default_rng(6).integers(0, len(rec), 512)
    blob = I.workload_weights(I.Workload("t", ARCH, 1, 1, seed=5))
    cfg = oracle.Config.of(ARCH)
    x = oracle_windows(rec, L, idx)
    y = np.stack([L.F[idx], L.E[idx]], 1).astype(np.float64)
    loss_o, g_o = oracle.loss_grad(cfg, blob, x, y)
    theta, m, v = blob.astype(np.float32).astype(np.float64), np.zeros_like(blob), np.zeros_like(blob)
    oracle.adam(theta, m, v, g_o, lr=1e-3, t=1)
    sim, _ = make_sim(ARCH, precision, blob=blob)
    loss = sim.train_step(w, torch.from_numpy(idx).cuda(), lr=1e-3)
    new = sim.get_weights().astype(np.float64)
    tol = 1e-4 if precision == "fp32" else 2e-2
    assert loss == pytest.approx(loss_o, rel=tol)
    d_gpu, d_or = new - blob.astype(np.float32), theta - blob.astype(np.float32)
    sure = np.abs(g_o) > 1e-3 * np.abs(g_o).max()        # Adam's first step is lr * sign(g)
    frac = np.mean(np.abs(d_gpu[sure] - d_or[sure]) < 1e-4)
    assert frac > (0.999 if precision == "fp32" else 0.97), frac


def test_training_reduces_loss_and_tracks_autograd(data):
    """Library-fused Adam steps vs the same model trained through CNNFunction
    with torch.optim.Adam from the same initial weights and batches."""
    rec, L, w = data
    blob = I.workload_weights(I.Workload("t", ARCH, 1, 1, seed=6)).astype(np.float32)
    a, _ = make_sim(ARCH, "fp32", blob=blob)
    b, _ = make_sim(ARCH, "fp32", blob=blob)
    wt = torch.from_numpy(blob).cuda().requires_grad_(True)
    opt = torch.optim.Adam([wt], lr=1e-3)
    gen = torch.Generator(device="cuda").manual_seed(1)
    la, lb = [], []
    for s in range(100):
        idx = torch.randint(0, len(w), (256,), device="cuda", generator=gen)
        la.append(a.train_step(w, idx, 1e-3))
        x = b.gather_windows(w, idx)
        opt.zero_grad()
        loss = LossFunction.apply(CNNFunction.apply(x, wt, b), w.labels[idx], b)
        loss.backward()
        opt.step()
        lb.append(loss.item())
    la, lb = np.array(la), np.array(lb)
    assert np.abs(la[:10] - lb[:10]).max() / lb[0] < 1e-3
    assert la[-10:].mean() < 0.7 * la[:3].mean()       # labels up to 255 cycles: slow at lr 1e-3

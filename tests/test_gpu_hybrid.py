"""GPU parity of the hybrid latency head (Sec. 2.3): per latency ten class
logits (0..8 cycles and "more than 8") plus a regression output that the last
class uses, trained with cross-entropy + squared error.

* Decisions the network cannot blur: with FC2's weights at zero the outputs
  equal the biases, so every decision (direct classes, ties, class 9 through
  the regression output) is known exactly; every kernel path must take it.
* Real networks: integer state bit-exact under teacher forcing both ways,
  regression outputs within the precision's bound, FC2 outputs against the
  oracle's, and each free-running decision equal to the oracle's decision on
  the same state wherever the logit margin exceeds the precision's error.
* Training: loss, gradient and one Adam step against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import SimnetError
from paper_2105_05821_b300.train import CNNFunction, LossFunction, Windows

from gpu_util import hybrid_loss, latency_error, make_sim, run_gpu
from test_gpu_sim import teacher_forced_check
from test_oracle_hybrid import bias_only_blob
from tolerances import check


def sim_windows(arch, blob, n, seed):
    """n feature matrices the simulator builds: the oracle's per-step inputs on
    a short synthetic trace with these weights."""
    trace = I.small_trace([n // 3, n // 3, n - 2 * (n // 3)], seed=seed)
    return oracle.simulate(oracle.Config.of(arch), trace.records, trace.offsets, blob, features=True).feat

pytestmark = pytest.mark.gpu


def hyb(arch: I.Arch) -> I.Arch:
    return I.Arch(arch.window, arch.n_conv, arch.channels, arch.hidden, "hybrid")


ARCH = hyb(I.ARCH_SMALL(32))       # every kernel path takes it (cluster: BF16, 2 x Conv64, FC256)

# (precision, Simnet keyword arguments, expected kernel path)
PATHS = {
    "fp32": ("fp32", {}, "layerwise"),
    "bf16-layerwise": ("bf16", {"persistent": False}, "layerwise"),
    "bf16-persistent": ("bf16", {"cluster": False}, "persistent"),
    "bf16-cluster": ("bf16", {}, "cluster"),
    "fp8-layerwise": ("fp8", {"persistent": False}, "layerwise"),
    "fp8-persistent": ("fp8", {"cluster": False}, "persistent"),
    "fp8-cluster": ("fp8", {}, "cluster"),
}
# precision -> smallest share of decisions whose margin exceeds the GPU's error
# (the latency bounds are the precision rows of tests/tolerances.py)
MIN_CLEAR = {"fp32": 0.95, "bf16": 0.5, "fp8": 0.2}


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("case", ["direct", "ties", "more_than_8"])
def test_bias_only_decisions_exact(path, case):
    precision, kw, kind = PATHS[path]
    lf, le = np.zeros(10), np.zeros(10)
    if case == "direct":          # fetch class 3; execution "more than 8" with softplus(2) = 2.13 -> 2
        lf[3], le[9] = 2.0, 5.0
        vf, ve, expect = -50.0, 2.0, (3, 2)
    elif case == "ties":          # exact tie -> the lower class, 2; 2^-20 apart (exact in FP32) -> class 5
        lf[2] = lf[6] = 1.5
        le[4], le[5] = 1.0, 1.0 + 2.0 ** -20
        vf, ve, expect = 0.0, 0.0, (2, 5)
    else:                         # both "more than 8": softplus(0.3) = 0.85 -> 1, softplus(12) -> 12
        lf[9], le[9] = 1.0, 1.0
        vf, ve, expect = 0.3, 12.0, (1, 12)
    blob = bias_only_blob(ARCH, lf, vf, le, ve)
    trace = I.small_trace([40, 7, 1, 0, 130, 64], seed=3)
    sim, _ = make_sim(ARCH, precision, blob=blob, **kw)
    g = run_gpu(sim, trace)
    assert sim.kernel_path == kind
    assert (g["lat"][:, 0] == expect[0]).all() and (g["lat"][:, 1] == expect[1]).all()
    ref = oracle.simulate(oracle.Config.of(ARCH), trace.records, trace.offsets, blob, logs=True)
    np.testing.assert_array_equal(ref.lat, g["lat"])
    np.testing.assert_array_equal(ref.cycles, g["cycles"])


def decisions_check(sim, arch, blob, trace, free_lat, min_clear):
    """Each free-running GPU decision against the oracle's decision on the same
    state: the oracle replays the GPU's latencies, logging every step's features,
    and its head decides on its own FP64 FC2 outputs for them.  A decision must
    match where its margin (gap between the two largest logits; for "more than
    8", also the distance of softplus(value) from a rounding boundary) exceeds
    three times the GPU's own FC2 error on that state (the library's CNN on the
    same features at the context's precision)."""
    cfg = oracle.Config.of(arch)
    back = oracle.simulate(cfg, trace.records, trace.offsets, replay=free_lat, logs=True, features=True)
    z = oracle.cnn_forward(cfg, blob, back.feat)
    lat_o, pre_o = oracle.head(cfg, z)
    zg = sim.cnn_forward(torch.from_numpy(back.feat.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    clear = np.ones(free_lat.shape, bool)
    for t in range(2):
        lg = z[:, 11 * t:11 * t + 10]
        err = np.abs(zg[:, 11 * t:11 * t + 10] - z[:, 11 * t:11 * t + 10]).max(1)
        top = np.sort(lg, 1)
        clear[:, t] = (top[:, -1] - top[:, -2]) > 3.0 * err + 1e-5 * (np.abs(lg).max(1) + 1.0)
        more = lat_o[:, t] > 8
        frac = pre_o[:, t] - np.floor(pre_o[:, t])
        perr = np.abs(oracle.softplus(zg[:, 11 * t + 10]) - pre_o[:, t])
        clear[more, t] &= np.abs(frac[more] - 0.5) > 3.0 * perr[more] + 1e-5 * (pre_o[more, t] + 1.0)
    assert clear.mean() >= min_clear, clear.mean()
    bad = np.argwhere(clear & (free_lat != lat_o))
    assert len(bad) == 0, (len(bad), bad[:5], z[bad[0][0]] if len(bad) else None)
    return clear.mean()


@pytest.mark.parametrize("path", list(PATHS))
def test_real_network_teacher_forced_and_decisions(path):
    precision, kw, kind = PATHS[path]
    min_clear = MIN_CLEAR[precision]
    blob = I.workload_weights(I.Workload("h", ARCH, 1, 1, seed=7))
    trace = I.small_trace([300, 130, 77, 0, 1, 45], seed=5)
    ref, free, err = teacher_forced_check(ARCH, trace, precision, blob, path=kind, **kw)
    assert (ref.lat[:, 1] > 8).any() and (ref.lat[:, 1] <= 8).any()   # both kinds of decision occur
    sim, _ = make_sim(ARCH, precision, blob=blob, **kw)
    decisions_check(sim, ARCH, blob, trace, free["lat"], min_clear)


def test_c2_architecture_hybrid_cluster():
    """The headline CNN shape (W=96, 3 x Conv128, FC512; 8-CTA clusters)."""
    arch = hyb(I.ARCH_MID)
    blob = I.workload_weights(I.Workload("h", arch, 1, 1, seed=2))
    trace = I.small_trace([400, 37, 250, 0, 128], seed=21)
    ref, free, _ = teacher_forced_check(arch, trace, "bf16", blob, path="cluster")
    sim, _ = make_sim(arch, "bf16", blob=blob)
    decisions_check(sim, arch, blob, trace, free["lat"], MIN_CLEAR["bf16"])


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_cnn_forward_outputs(precision):
    """FC2 outputs, element by element, on the feature rows the simulator
    builds (the oracle's per-step inputs of a short trace)."""
    cfg = oracle.Config.of(ARCH)
    blob = I.workload_weights(I.Workload("h", ARCH, 1, 1, seed=7))
    x = sim_windows(ARCH, blob, 300, seed=12)
    sim, _ = make_sim(ARCH, precision, blob=blob)
    z = sim.cnn_forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    zr = oracle.cnn_forward(cfg, blob, x)
    assert z.shape == (300, 22)
    check(latency_error(z, zr), precision, "hybrid CNN outputs, element by element")
    if precision == "fp32":
        zn = torch.empty((300, 22), dtype=torch.float32, device="cuda")
        sim.cnn_forward_noalloc(torch.from_numpy(x.astype(np.float32)).cuda(), zn)
        check(latency_error(zn.cpu().numpy(), zr), precision, "hybrid CNN outputs, no-allocation entry point")


@pytest.fixture(scope="module")
def data():
    rec = I.make_records(6000, 33)
    L = I.toy_labels(rec)
    return rec, L, Windows.from_labels(rec, L)


def test_training_gradient_and_adam_match_oracle(data):
    rec, L, w = data
    arch = hyb(I.ARCH_SMALL(96))
    cfg = oracle.Config.of(arch)
    idx = np.random.default_rng(5).integers(0, len(rec), 256)
    blob = I.workload_weights(I.Workload("t", arch, 1, 1, seed=3))
    x = oracle.window_features(cfg, rec, L.fetch, L.E, L.ctx_begin, idx)
    y = np.stack([L.F[idx], L.E[idx]], 1).astype(np.float64)
    loss_o, g_o = oracle.loss_grad(cfg, blob, x, y)
    # autograd through the library's forward/backward with the torch loss
    sim, _ = make_sim(arch, "fp32", blob=blob)
    wt = torch.from_numpy(blob.astype(np.float32)).cuda().requires_grad_(True)
    z = CNNFunction.apply(torch.from_numpy(x.astype(np.float32)).cuda(), wt, sim)
    assert tuple(z.shape) == (256, 22)
    loss = LossFunction.apply(z, torch.from_numpy(y.astype(np.uint8)).cuda(), sim)   # the library's loss kernel
    loss.backward()
    assert loss.item() == pytest.approx(hybrid_loss(z.detach().double(), torch.from_numpy(y).cuda()).item(),
                                        rel=1e-5)
    assert loss.item() == pytest.approx(loss_o, rel=1e-4)
    g = wt.grad.cpu().numpy().astype(np.float64)
    k = 0
    for name, shape in arch.shapes():
        n = int(np.prod(shape))
        rel = np.linalg.norm(g[k:k + n] - g_o[k:k + n]) / max(np.linalg.norm(g_o[k:k + n]), 1e-30)
        assert rel < 1e-3, (name, rel)
        k += n
    # the fused step: the library's own hybrid loss, backward and Adam
    theta, m, v = blob.astype(np.float32).astype(np.float64), np.zeros_like(blob), np.zeros_like(blob)
    oracle.adam(theta, m, v, g_o, lr=1e-3, t=1)
    fused, _ = make_sim(arch, "fp32", blob=blob)
    lf = fused.train_step(w, torch.from_numpy(idx).cuda(), lr=1e-3)
    assert lf == pytest.approx(loss_o, rel=1e-4)
    d_gpu, d_or = fused.get_weights().astype(np.float64) - blob.astype(np.float32), theta - blob.astype(np.float32)
    sure = np.abs(g_o) > 1e-3 * np.abs(g_o).max()
    assert np.mean(np.abs(d_gpu[sure] - d_or[sure]) < 1e-4) > 0.999


def test_training_reduces_hybrid_loss(data):
    rec, L, w = data
    arch = hyb(I.ARCH_SMALL(96))
    sim, _ = make_sim(arch, "bf16", blob=I.workload_weights(I.Workload("t", arch, 1, 1, seed=6)))
    gen = torch.Generator(device="cuda").manual_seed(1)
    losses = [sim.train_step(w, torch.randint(0, len(w), (256,), device="cuda", generator=gen), 1e-3)
              for _ in range(60)]
    assert np.isfinite(losses).all() and np.mean(losses[-10:]) < 0.8 * np.mean(losses[:3])


def test_state_of_the_other_head_is_refused():
    blob_h = I.workload_weights(I.Workload("h", ARCH, 1, 1, seed=7))
    a, _ = make_sim(ARCH, "fp32", blob=blob_h)
    st = a.state_save("train")
    reg = I.ARCH_SMALL(32)
    b, _ = make_sim(reg, "fp32")
    with pytest.raises(SimnetError):
        b.state_load(st, "train")
    c, _ = make_sim(ARCH, "fp32", blob=np.zeros_like(blob_h))
    c.state_load(st, "train")
    np.testing.assert_array_equal(c.get_weights(), blob_h.astype(np.float32))

"""GPU parity of the residual-block CNN (the RB models of Sec. 2.3; block k:
a = ReLU(conv(x)), y = ReLU(pw(a) + proj(x))) against the FP64 oracle, whose
forward pass is pinned to PyTorch float64 on the CPU.

A block is three GEMMs (the conv, the bias-free projection shortcut, and the
pointwise conv whose epilogue adds the shortcut before the ReLU), run as
per-layer kernels (FP32, or BF16 with SIMNET_FLAG_LAYERWISE) or as phases of
the grid-persistent kernel (BF16 default), which computes only the positions
below the padding extent: the pointwise phase reads and writes the pair-major
tiles as rows of positions, and the padding table follows the constant row
through every block.  Integer state bit-exact under teacher forcing both ways;
outputs within the precision's bound; the two BF16 paths agree on identical
states; the RB7 shape (W=128, 7 blocks of 256 channels, FC1024, hybrid head)
included.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import Simnet, SimnetError

from gpu_util import latency_error, make_sim, run_gpu
from test_gpu_sim import teacher_forced_check
from test_gpu_hybrid import sim_windows
from tolerances import LAT_MAX, check

pytestmark = pytest.mark.gpu


def rb(arch: I.Arch, head: str = "regression") -> I.Arch:
    return I.Arch(arch.window, arch.n_conv, arch.channels, arch.hidden, head, block="residual")


SMALL = rb(I.Arch(32, 3, 64, 256))
PATHS = {"fp32": ("fp32", {}, "layerwise"), "bf16-layerwise": ("bf16", {"persistent": False}, "layerwise"),
         "bf16-persistent": ("bf16", {}, "persistent")}


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("head", ["regression", "hybrid"])
def test_small_residual_network(path, head):
    precision, kw, kind = PATHS[path]
    arch = rb(I.Arch(32, 3, 64, 256), head)
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=3))
    trace = I.small_trace([0, 1, 5, 33, 130, 7, 64, 0, 250], seed=9)
    ref, free, err = teacher_forced_check(arch, trace, precision, blob, path=kind, **kw)
    assert np.isfinite(free["pre"]).all()


@pytest.mark.parametrize("path", list(PATHS))
def test_rb7_shape(path):
    precision, kw, kind = PATHS[path]
    w = I.WORKLOADS["rb7"]
    blob = I.workload_weights(w)
    trace = I.small_trace([120, 90, 0, 60, 1, 100, 75, 110], seed=13)
    teacher_forced_check(w.arch, trace, precision, blob, path=kind, **kw)


@pytest.mark.parametrize("arch", [SMALL, I.WORKLOADS["rb7"].arch])
def test_persistent_matches_per_layer_on_identical_states(arch):
    """The padding-extent kernel against the dense per-layer kernels, both
    replaying the oracle's latencies (identical states): identical integer
    state, regression outputs equal to BF16 rounding."""
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=8))
    lengths = np.clip(np.rint(np.exp(np.random.default_rng(2).normal(np.log(80), 0.7, 200))), 1, 300).astype(int)
    trace = I.small_trace(lengths.tolist(), seed=17)
    lw, _ = make_sim(arch, "bf16", blob=blob, persistent=False)
    ps, _ = make_sim(arch, "bf16", blob=blob)
    replay = np.stack([np.random.default_rng(3).integers(0, 3, trace.n_instructions),
                       np.random.default_rng(4).integers(0, 20, trace.n_instructions)], 1).astype(np.uint8)
    g = run_gpu(lw, trace, replay=replay)
    h = run_gpu(ps, trace, replay=replay)
    assert ps.kernel_path == "persistent" and lw.kernel_path == "layerwise"
    np.testing.assert_array_equal(h["cycles"], g["cycles"])
    d = latency_error(h["pre"], g["pre"])
    assert np.median(d) < 1e-3 and d.max() < 2 * LAT_MAX["bf16"], (np.median(d), d.max())


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_cnn_forward_outputs(precision):
    arch = rb(I.Arch(32, 3, 64, 256), "hybrid")
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=5))
    x = sim_windows(arch, blob, 200, seed=4)   # the feature rows the simulator builds
    sim, _ = make_sim(arch, precision, blob=blob)
    z = sim.cnn_forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    zr = oracle.cnn_forward(oracle.Config.of(arch), blob, x)
    assert z.shape == (200, 22)
    check(latency_error(z, zr), precision, "residual CNN outputs, element by element")


def test_unsupported_modes_are_refused():
    with pytest.raises(SimnetError):
        Simnet.for_arch(SMALL, precision="fp8")
    from paper_2105_05821_b300.train import Windows
    rec = I.make_records(500, 3)
    w = Windows.from_labels(rec, I.toy_labels(rec))
    sim, blob = make_sim(SMALL, "bf16")
    with pytest.raises(SimnetError):
        sim.train_step(w, torch.arange(64, device="cuda"), 1e-3)
    with pytest.raises(SimnetError):
        sim.cnn_forward_noalloc(torch.zeros((4, 32, 50), device="cuda"), torch.zeros((4, 2), device="cuda"))
    np.testing.assert_array_equal(sim.get_weights(), blob.astype(np.float32))

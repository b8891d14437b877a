"""GPU parity of the residual-block CNN (the RB models of Sec. 2.3; block k:
a = ReLU(conv(x)), y = ReLU(pw(a) + proj(x))) against the FP64 oracle, whose
forward pass is pinned to PyTorch float64 on the CPU.

Residual networks run as per-layer kernels: three GEMMs a block (the conv, the
bias-free projection shortcut, and the pointwise conv whose epilogue adds the
shortcut before the ReLU), FC1 with FC2 folded in, then the head and queue
update.  Integer state bit-exact under teacher forcing both ways; outputs
within the precision's bound; the RB7 shape (W=128, 7 blocks of 256 channels,
FC1024, hybrid head) included.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import Simnet, SimnetError

from gpu_util import make_sim, run_gpu
from test_gpu_sim import teacher_forced_check

pytestmark = pytest.mark.gpu


def rb(arch: I.Arch, head: str = "regression") -> I.Arch:
    return I.Arch(arch.window, arch.n_conv, arch.channels, arch.hidden, head, block="residual")


SMALL = rb(I.Arch(32, 3, 64, 256))
TOL = {"fp32": 1e-3, "bf16": 5e-2}


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("head", ["regression", "hybrid"])
def test_small_residual_network(precision, head):
    arch = rb(I.Arch(32, 3, 64, 256), head)
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=3))
    trace = I.small_trace([0, 1, 5, 33, 130, 7, 64, 0, 250], seed=9)
    ref, free, err = teacher_forced_check(arch, trace, precision, blob, TOL[precision], path="layerwise")
    assert ref.evictions.sum() >= 0 and np.isfinite(free["pre"]).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rb7_shape(precision):
    w = I.WORKLOADS["rb7"]
    blob = I.workload_weights(w)
    trace = I.small_trace([120, 90, 0, 60, 1, 100, 75, 110], seed=13)
    teacher_forced_check(w.arch, trace, precision, blob, TOL[precision], path="layerwise")


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 3e-2)])
def test_cnn_forward_outputs(precision, tol):
    arch = rb(I.Arch(32, 3, 64, 256), "hybrid")
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=5))
    x = I.random_windows(200, arch, 4)
    sim, _ = make_sim(arch, precision, blob=blob)
    z = sim.cnn_forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    zr = oracle.cnn_forward(oracle.Config.of(arch), blob, x)
    assert z.shape == (200, 22)
    assert np.abs(z - zr).max() / (np.abs(zr).max() + 1.0) < tol


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

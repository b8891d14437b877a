"""GPU parity of the FP8 e4m3 tensor-core path against the FP64 oracle.

Integer state stays bit-exact under teacher forcing.  Predicted latencies carry
e4m3 rounding (3 mantissa bits) of features, weights and activations, with
per-output-channel weight scales and calibrated per-channel activation scales
folded into the next layer's weights; the asserted bounds are the FP8 row of
tests/tolerances.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I

from gpu_util import latency_error, make_sim, run_gpu
from test_gpu_sim import teacher_forced_check
from test_gpu_tc import real_windows
from tolerances import check, check_cpi

pytestmark = pytest.mark.gpu



@pytest.mark.parametrize("arch", [I.ARCH_SMALL(32), I.ARCH_MID, I.ARCH_WIDE, I.ARCH_SMALL(96)])
def test_cnn_forward_fp8(arch):
    x, blob = real_windows(arch, seed=arch.window + arch.n_conv)
    sim, _ = make_sim(arch, "fp8", blob=blob)
    z = sim.cnn_forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    zr = oracle.cnn_forward(oracle.Config.of(arch), blob, x)
    assert np.isfinite(z).all()
    check(latency_error(oracle.softplus(z), oracle.softplus(zr)), "fp8", f"latencies {arch}")
    check(latency_error(z, zr), "fp8", f"CNN outputs {arch}")


def test_c1_fp8_teacher_forced():
    w = I.WORKLOADS["c1"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    ref, free, err = teacher_forced_check(w.arch, trace, "fp8", blob)
    check_cpi(abs(free["cycles"].sum() / ref.cycles.sum() - 1.0), "fp8", "c1 free-running")


def test_c2_full_size_sampled_fp8():
    w = I.WORKLOADS["c2"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    sim, _ = make_sim(w.arch, "fp8", blob=blob)
    g = run_gpu(sim, trace)
    ids = [0, 3, 300, 777, 1023]
    cfg = oracle.Config.of(w.arch)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, blob, subset=ids, replay=g["lat"], logs=True)
    np.testing.assert_array_equal(ref.cycles, g["cycles"][ids])
    sel = np.concatenate([np.arange(trace.offsets[i], trace.offsets[i + 1]) for i in ids])
    check(latency_error(g["pre"][sel], ref.pre[sel]), "fp8", "c2 full size, 5 sampled sub-traces")
    free = oracle.simulate(cfg, trace.records, trace.offsets, blob, subset=ids)
    check_cpi(abs(g["cycles"][ids].sum() / free.cycles.sum() - 1.0), "fp8", "c2, 5 sampled sub-traces")

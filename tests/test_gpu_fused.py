"""The persistent kernel's fused first two conv layers (a plain CNN of 256
channels): one phase computes each tile of conv2's output from conv1's two
positions under it, and conv1's output stays in tensor memory as conv2's A
operand instead of going through device memory (Sec. 2.3's k=2 / stride-2
convolutions, composed).

* Against the FP64 oracle under teacher forcing both ways: integer state
  bit-exact, predicted latencies within the precision's row, BF16 and FP8, on
  a ragged batch and an uneven one (three slot blocks, the last partial,
  compaction), at W=32 and at the c5 shape (W=128, 5 x Conv256, FC1024).
* Against the same kernel with the fusion off (conv1's output through device
  memory) on identical states: the same cycle counts and the same predicted
  latencies, value for value, since both round conv1's output the same way
  and accumulate conv2 over K in the same order.
* The phase timing shows which ran: no conv1 phase when fused.
"""
import numpy as np
import pytest

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import KERNEL_LAYER0

from gpu_util import latency_error, make_sim, run_gpu
from tolerances import check

pytestmark = pytest.mark.gpu

SMALL = I.Arch(32, 3, 256, 512)


def case_inputs(case):
    if case == "c5arch":
        w = I.WORKLOADS["c5"]
        return w.arch, I.small_trace([260, 37, 150, 0, 64, 3], seed=23), I.workload_weights(w)
    if case == "ragged":
        lengths = [0, 1, 5, 33, 130, 7, 64, 0]
    else:
        lengths = np.clip(np.rint(np.exp(np.random.default_rng(9).normal(np.log(30), 0.7, 300))), 1, 200)
        lengths = lengths.astype(int).tolist()
    blob = I.workload_weights(I.Workload("fused", SMALL, 1, 1, seed=11))
    return SMALL, I.small_trace(lengths, seed=len(lengths) + 1), blob


def phase_counts(sim):
    _, n = sim.kernel_times()
    return n[KERNEL_LAYER0], n[KERNEL_LAYER0 + 1]


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("case", ["ragged", "uneven", "c5arch"])
def test_fused_conv_pair(precision, case):
    arch, trace, blob = case_inputs(case)
    cfg = oracle.Config.of(arch)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, blob, logs=True)
    fused, _ = make_sim(arch, precision, blob=blob, cluster=False)
    plain, _ = make_sim(arch, precision, blob=blob, cluster=False, fuse=False)
    # teacher forcing with the oracle's latencies: integers exact, latencies within the row
    h = run_gpu(fused, trace, replay=ref.lat)
    assert fused.kernel_path == "persistent"
    np.testing.assert_array_equal(h["cycles"], ref.cycles)
    np.testing.assert_array_equal(h["lat"], ref.lat)
    assert np.isfinite(h["pre"]).all()
    check(latency_error(h["pre"], ref.pre), precision, f"fused conv pair, {case}")
    # the unfused phases on the same states give the same values
    g = run_gpu(plain, trace, replay=ref.lat)
    assert plain.kernel_path == "persistent"
    np.testing.assert_array_equal(g["cycles"], h["cycles"])
    np.testing.assert_array_equal(g["pre"], h["pre"])
    # free running: the oracle replays the fused kernel's own latencies
    f = run_gpu(fused, trace)
    back = oracle.simulate(cfg, trace.records, trace.offsets, replay=f["lat"], logs=True)
    np.testing.assert_array_equal(back.cycles, f["cycles"])


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_fused_phase_replaces_conv1_phase(precision):
    arch, trace, blob = case_inputs("ragged")
    counts = {}
    for fuse in (True, False):
        sim, _ = make_sim(arch, precision, blob=blob, cluster=False, fuse=fuse, kernel_events=True)
        run_gpu(sim, trace, logs=False)
        assert sim.kernel_path == "persistent"
        counts[fuse] = phase_counts(sim)
    assert counts[True][0] == 0 and counts[True][1] > 0, counts
    assert counts[False][0] > 0 and counts[False][1] == counts[False][0], counts
    assert counts[True][1] == counts[False][1], counts

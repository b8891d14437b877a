"""GPU parity at the benchmark's largest sizes, in the launch configuration
`bench.py` times (default flags: the library picks its kernel path).

* c5: 65,536 sub-traces x ~1,526 instructions (100M), W=128, 5 x Conv256,
  FC1024, BF16 and FP8.
* c4: 4,096 log-normal sub-traces (about 40M instructions) with the trained
  c2-architecture predictor (300 fused Adam steps on toy-pipeline labels, as
  the benchmark trains it), BF16 and FP8.  Its queues stay long, so a BF16
  call starts on the cluster kernel and hands the batch to the grid-wide path
  after the probe; the cycle counts must not notice.

The oracle cannot run 100M instructions, so each test samples sub-traces
(independent by construction, Sec. 3.3), re-simulates them with the GPU's own
latencies (cycle counts bit-exact) and compares the GPU's predicted latencies
on those states with the oracle's (the precision's row of tests/tolerances.py),
then runs them free (CPI error within the row).
"""
import sys
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I

from gpu_util import latency_error, make_sim, to_dev
from tolerances import check, check_cpi

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

pytestmark = pytest.mark.gpu


def extract(trace: I.Trace, ids):
    """The listed sub-traces as a trace of their own, and the global positions
    of their instructions."""
    sel = np.concatenate([np.arange(trace.offsets[i], trace.offsets[i + 1]) for i in ids])
    lens = np.array([trace.offsets[i + 1] - trace.offsets[i] for i in ids])
    return I.Trace(trace.records[sel].copy(), np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)), sel


def sampled_check(w, trace, blob, precision, ids, expect_paths):
    sim, _ = make_sim(w.arch, precision, blob=blob, retire_width=w.retire_width, auto_path=True)
    rec, off = to_dev(trace)
    N, NL = trace.n_instructions, sim.n_lat
    lat = torch.zeros((N, NL), dtype=torch.uint8, device="cuda")
    pre = torch.full((N, NL), float("nan"), dtype=torch.float32, device="cuda")
    sim.simulate(rec, off, lat_log=lat, pre_log=pre)
    torch.cuda.synchronize()
    assert sim.kernel_path in expect_paths, sim.kernel_path
    cycles = sim.cycles.cpu().numpy()
    small, sel = extract(trace, ids)
    sel_t = torch.from_numpy(sel).cuda()
    lat_s, pre_s = lat[sel_t].cpu().numpy(), pre[sel_t].cpu().numpy()
    del lat, pre
    sim.close()
    cfg = oracle.Config.of(w.arch, retire_width=w.retire_width)
    back = oracle.simulate(cfg, small.records, small.offsets, blob, replay=lat_s, logs=True)
    np.testing.assert_array_equal(back.cycles, cycles[ids])
    check(latency_error(pre_s, back.pre), precision, f"{w.name} full size, {len(ids)} sampled sub-traces")
    free = oracle.simulate(cfg, small.records, small.offsets, blob)
    check_cpi(abs(cycles[ids].sum() / free.cycles.sum() - 1.0), precision,
              f"{w.name} full size, {len(ids)} sampled sub-traces")
    return cycles


@pytest.fixture(scope="module")
def c5():
    w = I.WORKLOADS["c5"]
    return w, I.make_trace(w), I.workload_weights(w)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_c5_full_size_sampled(c5, precision):
    w, trace, blob = c5
    assert trace.n_subtraces == 65_536 and trace.n_instructions == 100_000_000
    ids = sorted(np.random.default_rng(50).choice(trace.n_subtraces, 8, replace=False).tolist())
    ids[0], ids[-1] = 0, trace.n_subtraces - 1          # the first and the last sub-trace too
    sampled_check(w, trace, blob, precision, ids, ("persistent", "layerwise"))


@pytest.fixture(scope="module")
def c4():
    w = I.WORKLOADS["c4"]
    blob32, info = bench.train_predictor(w, 300)
    return w, I.make_trace(w), blob32.astype(np.float64), info


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_c4_full_size_trained_sampled(c4, precision):
    w, trace, blob, info = c4
    assert trace.n_subtraces == 4096 and info["loss_last"] < info["loss_first"]
    ids = sorted(np.random.default_rng(40).choice(trace.n_subtraces, 8, replace=False).tolist())
    # BF16 starts on the cluster kernel; the probe sees long queues and hands over
    sampled_check(w, trace, blob, precision, ids, ("persistent", "layerwise"))

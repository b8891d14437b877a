"""Randomised parity of the integer state machine on every GPU kernel path.

Each case draws a CNN shape, a retire width and rule, ragged sub-trace lengths
(empty, single-instruction and long ones mixed), a precision and a kernel path,
and replays seeded random latencies F, E (Sec. 3.2): the CNN's outputs are
then irrelevant, so the per-sub-trace cycle counts, the evictions and the
logged latencies must equal the oracle's bit for bit on the cluster kernel,
the grid-persistent kernel, the per-layer kernels and the FP32 form alike, for
the regression and hybrid heads, residual blocks and (with a third, store
latency) the memory write queue.
The latency mixes cover an empty retire budget (F = 0), queues that overflow
(long E) and queues that stay short.  Each case is run again in bounded calls
of random lengths (the resumable state carried between them) and must give
the same run.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I

from gpu_util import make_sim, run_gpu, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [I.ARCH_SMALL(32), I.ARCH_MID]
# (precision, Simnet keyword arguments, kernel path the call must report)
PATHS = [
    ("bf16", {}, "cluster"),
    ("bf16", {"cluster": False}, "persistent"),
    ("bf16", {"persistent": False}, "layerwise"),
    ("fp8", {}, "cluster"),
    ("fp8", {"cluster": False}, "persistent"),
    ("fp8", {"persistent": False}, "layerwise"),
    ("fp32", {}, "layerwise"),
]


def latencies(rng, n, mix):
    if mix == "short":      # queues stay short: everything retires within a few steps
        f, e = rng.integers(1, 4, n), rng.integers(0, 6, n)
    elif mix == "overflow":  # F = 1, long E: queues fill to capacity and evict
        f, e = np.ones(n, np.int64), rng.integers(100, 256, n)
    else:                   # F = 0 in a third of the steps (no retire budget), wide E
        f, e = rng.integers(0, 3, n), rng.integers(0, 60, n)
    return np.stack([f, e], 1).astype(np.uint8)


HYBRID = I.Arch(96, 3, 128, 512, "hybrid")               # 22 FC2 outputs: other kernel instances
STORE = I.Arch(32, 2, 64, 256, store_queue=True)          # three latencies, memory write queue
RESID = I.Arch(32, 2, 64, 256, block="residual")          # residual blocks: BF16 and FP32 only
CASES = ([(a, p) for a in SHAPES for p in PATHS] + [(HYBRID, p) for p in PATHS]
         + [(STORE, p) for p in PATHS]
         + [(RESID, p) for p in PATHS if p[0] != "fp8" and p[2] != "cluster"])


def latencies3(rng, n, mix):
    s = rng.integers(0, 80, n) if mix != "short" else rng.integers(0, 6, n)
    return np.concatenate([latencies(rng, n, mix), s[:, None].astype(np.uint8)], 1)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_random_replay_bit_exact(case):
    rng = np.random.default_rng(1000 + case)
    arch, (precision, kw, path) = CASES[case]
    rw, strict = int(rng.integers(1, 9)), bool(rng.integers(0, 2))
    n_sub = int(rng.choice([3, 40, 200]))
    lengths = rng.integers(0, 400, n_sub)
    lengths[rng.random(n_sub) < 0.1] = 0
    lengths[rng.random(n_sub) < 0.1] = 1
    trace = I.small_trace(lengths.tolist(), seed=2000 + case)
    mix = ["short", "overflow", "mixed"][case % 3]
    replay = (latencies3 if arch.store_queue else latencies)(rng, trace.n_instructions, mix)
    cfg = oracle.Config.of(arch, retire_width=rw, retire_strict=strict)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, replay=replay, logs=True)
    sim, _ = make_sim(arch, precision, retire_width=rw, strict=strict, **kw)
    g = run_gpu(sim, trace, replay=replay)
    assert sim.kernel_path == path
    np.testing.assert_array_equal(g["cycles"], ref.cycles)
    np.testing.assert_array_equal(g["lat"], ref.lat)
    assert g["stats"].evictions == int(ref.evictions.sum())
    assert g["stats"].total_cycles == int(ref.cycles.sum())
    # the same call in bounded pieces of random lengths (resumable state) gives the same run
    rec_d, off_d = to_dev(trace)
    rp = torch.from_numpy(np.ascontiguousarray(replay)).cuda()
    n = max(trace.n_instructions, 1)
    lat = torch.zeros((n, sim.n_lat), dtype=torch.uint8, device="cuda")
    cyc = torch.empty(trace.n_subtraces, dtype=torch.int64, device="cuda")
    resume, pending, calls = False, None, 0
    while pending != 0 and calls < 10000:
        st = sim.simulate(rec_d, off_d, cycles_out=cyc, lat_log=lat, replay=rp,
                          max_steps=int(rng.integers(1, 200)), resume=resume)
        pending, resume, calls = st.pending, True, calls + 1
    assert pending == 0
    np.testing.assert_array_equal(cyc.cpu().numpy(), ref.cycles)
    np.testing.assert_array_equal(lat.cpu().numpy()[:trace.n_instructions], ref.lat)

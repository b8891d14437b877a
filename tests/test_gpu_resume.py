"""Checkpoint / resume (lock-step loop of Sec. 3.3 and training of Sec. 2.4).

A simulation split into bounded calls, or saved, loaded into a fresh context
and resumed there, must give the unsplit run's cycle counts, integer latencies
and pre-rounding outputs bit for bit; a training state saved after k Adam steps
must load back byte for byte, and training resumed from it must track the
uninterrupted run.
The unsplit run itself is pinned to the FP64 oracle by the parity tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import SimnetError
from paper_2105_05821_b300.train import Windows

from gpu_util import make_sim, to_dev

pytestmark = pytest.mark.gpu

# uneven lengths (compaction runs mid-trace), an empty and a one-instruction sub-trace
LENGTHS = [0, 1, 37, 300, 41, 512, 90, 5, 260, 128, 64, 7, 1000, 3, 222, 99]
MODES = [("fp32", "layerwise"), ("bf16", "cluster"), ("bf16", "persistent"), ("bf16", "layerwise"),
         ("fp8", "cluster"), ("fp8", "persistent")]


def sim_for(arch, precision, mode, **kw):
    sim, blob = make_sim(arch, precision, persistent=mode != "layerwise", cluster=mode == "cluster", **kw)
    sim.mode = mode
    return sim, blob


def run(sim, rec, off, N, chunks=None, state_via=None):
    """Simulate to the end, in one call or in bounded calls of chunks[i] steps;
    state_via(sim) -> sim swaps contexts between calls through state bytes."""
    lat = torch.zeros((N, sim.n_lat), dtype=torch.uint8, device="cuda")
    pre = torch.full((N, sim.n_lat), float("nan"), dtype=torch.float32, device="cuda")
    cyc = torch.empty(off.numel() - 1, dtype=torch.int64, device="cuda")
    if chunks is None:
        st = sim.simulate(rec, off, cycles_out=cyc, lat_log=lat, pre_log=pre)
        assert st.pending == 0
    else:
        resume, k, pending = False, 0, None
        while pending != 0:
            st = sim.simulate(rec, off, cycles_out=cyc, lat_log=lat, pre_log=pre,
                              max_steps=chunks[k % len(chunks)], resume=resume)
            pending, resume, k = st.pending, True, k + 1
            if pending and state_via is not None:
                sim = state_via(sim)
        assert k > 2
    torch.cuda.synchronize()
    return cyc.cpu().numpy(), lat.cpu().numpy(), pre.cpu().numpy(), st


@pytest.fixture(scope="module")
def trace():
    return I.small_trace(LENGTHS, seed=11)


@pytest.mark.parametrize("precision,mode", MODES)
def test_split_run_equals_unsplit(trace, precision, mode):
    arch = I.ARCH_MID
    sim, blob = sim_for(arch, precision, mode, seed=3)
    rec, off = to_dev(trace)
    N = trace.n_instructions
    c0, l0, p0, st0 = run(sim, rec, off, N)
    c1, l1, p1, st1 = run(sim, rec, off, N, chunks=[1, 17, 64, 5])
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_array_equal(l1, l0)
    np.testing.assert_array_equal(p1.view(np.uint32), p0.view(np.uint32))
    assert st1.steps_done == max(LENGTHS) and st1.total_cycles == st0.total_cycles
    assert st1.evictions == st0.evictions
    assert sim.kernel_path == mode


@pytest.mark.parametrize("precision,mode", [("fp32", "layerwise"), ("bf16", "cluster"), ("bf16", "persistent")])
def test_saved_state_resumes_in_a_fresh_context(trace, precision, mode):
    arch = I.ARCH_SMALL(32)
    sim, blob = sim_for(arch, precision, mode, seed=5)
    rec, off = to_dev(trace)
    N = trace.n_instructions
    c0, l0, p0, _ = run(sim, rec, off, N)

    def move(old):
        data = old.state_save("sim")
        new, _ = sim_for(arch, precision, mode, blob=blob)
        new.state_load(data, "sim")
        old.close()
        return new

    c1, l1, p1, _ = run(sim, rec, off, N, chunks=[50, 9], state_via=move)
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_array_equal(l1, l0)
    np.testing.assert_array_equal(p1.view(np.uint32), p0.view(np.uint32))
    # the state carries finished sub-traces' cycles: check the split against the oracle too
    cfg = oracle.Config.of(arch)
    back = oracle.simulate(cfg, trace.records, trace.offsets, replay=l1, logs=False)
    np.testing.assert_array_equal(back.cycles, c1)


def test_resume_rejects_mismatches(trace):
    arch = I.ARCH_SMALL(32)
    sim, blob = make_sim(arch, "fp32", seed=5)
    rec, off = to_dev(trace)
    with pytest.raises(SimnetError, match="ESTATE"):
        sim.simulate(rec, off, max_steps=3, resume=True)            # nothing to resume
    st = sim.simulate(rec, off, max_steps=3)
    assert st.pending > 0 and st.steps == 3
    other = I.small_trace(LENGTHS[::-1], seed=11)
    r2, o2 = to_dev(other)
    with pytest.raises(SimnetError, match="ESTATE"):
        sim.simulate(r2, o2, max_steps=3, resume=True)              # another trace
    data = sim.state_save("sim")
    fresh, _ = make_sim(arch, "fp32", seed=6)                        # other weights
    fresh.state_load(data, "sim")
    with pytest.raises(SimnetError, match="ESTATE"):
        fresh.simulate(rec, off, resume=True)
    wrong, _ = make_sim(I.ARCH_SMALL(64), "fp32", seed=5)           # other window
    with pytest.raises(SimnetError, match="EINVAL"):
        wrong.state_load(data, "sim")
    bad = bytearray(data)
    bad[0:8] = b"NOTSTATE"
    with pytest.raises(SimnetError, match="EINVAL"):
        sim.state_load(bytes(bad), "sim")
    with pytest.raises(SimnetError, match="EINVAL"):
        sim.state_load(data[:-8], "sim")                             # truncated
    with pytest.raises(SimnetError, match="EINVAL"):
        sim.state_load(data, "train")                                # wrong kind
    # max_steps = 0 only initialises; the resumed run still completes
    st = sim.simulate(rec, off, max_steps=0)
    assert st.steps == 0 and st.pending == sum(1 for n in LENGTHS if n > 0)
    st = sim.simulate(rec, off, resume=True)
    assert st.pending == 0


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_training_state_round_trip(precision):
    """The saved training state loads back byte for byte; training continued
    from it tracks the uninterrupted run (weight gradients accumulate with
    float atomics, so two runs agree to rounding, not bit for bit)."""
    arch = I.ARCH_SMALL(96)
    rec = I.make_records(4000, 21)
    w = Windows.from_labels(rec, I.toy_labels(rec))
    gen = torch.Generator(device="cuda").manual_seed(2)
    batches = [torch.randint(0, len(w), (256,), device="cuda", generator=gen) for _ in range(10)]
    b, blob = make_sim(arch, precision, seed=8)
    for idx in batches[:4]:
        b.train_step(w, idx, 1e-3)
    data = b.state_save("train")
    c, _ = make_sim(arch, precision, seed=99)
    c.state_load(data, "train")
    assert c.state_save("train") == data
    for idx in batches[4:]:
        lb = b.train_step(w, idx, 1e-3)
        lc = c.train_step(w, idx, 1e-3)
        assert lc == pytest.approx(lb, rel=1e-4)
    wb, wc = b.get_weights(), c.get_weights()
    assert np.mean(np.abs(wb - wc) <= 1e-5 + 1e-4 * np.abs(wb)) > 0.999
    # a fresh optimiser (no saved moments) would not track it
    d, _ = make_sim(arch, precision, blob=blob)
    d.load_weights(np.frombuffer(data, np.float32, count=b.weight_count, offset=104).copy())
    for idx in batches[4:]:
        d.train_step(w, idx, 1e-3)
    assert np.mean(np.abs(wb - d.get_weights()) <= 1e-5 + 1e-4 * np.abs(wb)) < 0.9


@pytest.mark.parametrize("mode", ["cluster", "persistent"])
def test_bf16_padding_table_follows_device_weight_updates(trace, mode):
    """A BF16 context trained on the device simulates exactly as a fresh BF16
    context loaded with the trained weights (the single-launch kernels' table
    of padding-row FC1 sums is rebuilt from the updated masters)."""
    arch = I.ARCH_MID
    rec_t = I.make_records(3000, 4)
    w = Windows.from_labels(rec_t, I.toy_labels(rec_t))
    a, _ = sim_for(arch, "bf16", mode, seed=12)
    gen = torch.Generator(device="cuda").manual_seed(3)
    for _ in range(5):
        a.train_step(w, torch.randint(0, len(w), (128,), device="cuda", generator=gen), 1e-2)
    b, _ = sim_for(arch, "bf16", mode, blob=a.get_weights())
    rec, off = to_dev(trace)
    N = trace.n_instructions
    ca, la, pa, _ = run(a, rec, off, N)
    cb, lb, pb, _ = run(b, rec, off, N)
    np.testing.assert_array_equal(ca, cb)
    np.testing.assert_array_equal(la, lb)
    np.testing.assert_array_equal(pa.view(np.uint32), pb.view(np.uint32))


@pytest.mark.parametrize("variant", ["hybrid", "residual", "residual-hybrid"])
def test_split_run_equals_unsplit_other_networks(trace, variant):
    """Split runs on the grid-persistent kernel for the hybrid head and the
    residual network: every resumed launch starts from stale per-layer tiles and
    refills their constant rows, so the split run must still equal the unsplit
    one bit for bit."""
    base = I.ARCH_SMALL(32)
    head = "hybrid" if "hybrid" in variant else "regression"
    block = "residual" if "residual" in variant else "conv"
    arch = I.Arch(base.window, 3 if block == "residual" else base.n_conv, base.channels, base.hidden, head,
                  block=block)
    sim, blob = make_sim(arch, "bf16", seed=3, cluster=False)
    rec, off = to_dev(trace)
    N = trace.n_instructions
    c0, l0, p0, _ = run(sim, rec, off, N)
    c1, l1, p1, st1 = run(sim, rec, off, N, chunks=[1, 17, 64, 5])
    assert sim.kernel_path == "persistent"
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_array_equal(l1, l0)
    np.testing.assert_array_equal(p1.view(np.uint32), p0.view(np.uint32))
    back = oracle.simulate(oracle.Config.of(arch), trace.records, trace.offsets, replay=l1, logs=False)
    np.testing.assert_array_equal(back.cycles, c1)

"""GPU parity of the CUDA simulation path against the FP64 oracle.

Integer state (F/E, curTick, queue, cycle counts) must be bit-exact when both
sides use the same integer latencies (teacher forcing, both directions).  The
predicted latencies (softplus outputs before rounding) must agree within the
precision's row of tests/tolerances.py in the paper's error form
|f - y| / (y + 1) (FP32: 1e-3), and so must free-running CPI (FP32: 0.1 %).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import Simnet, SimnetError

from gpu_util import latency_error, make_sim, run_gpu
from tolerances import LAT_MAX, check, check_cpi

pytestmark = pytest.mark.gpu



def teacher_forced_check(arch, trace, precision, blob, rw=8, strict=False, graph=True, persistent=True,
                         cluster=True, path=None):
    cfg = oracle.Config.of(arch, retire_width=rw, retire_strict=strict)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, blob, logs=True)
    sim, _ = make_sim(arch, precision, blob=blob, retire_width=rw, strict=strict, graph=graph,
                      persistent=persistent, cluster=cluster)
    # GPU replays the oracle's latencies: every integer must match
    g = run_gpu(sim, trace, replay=ref.lat)
    if path is not None:
        assert sim.kernel_path == path
    np.testing.assert_array_equal(g["cycles"], ref.cycles)
    np.testing.assert_array_equal(g["lat"], ref.lat)
    assert g["stats"].evictions == int(ref.evictions.sum())
    assert g["stats"].total_cycles == int(ref.cycles.sum())
    err = latency_error(g["pre"], ref.pre)
    assert np.isfinite(g["pre"]).all()
    check(err, precision, f"teacher-forced latencies {arch}")
    # oracle replays the GPU's free-running latencies: every integer must match
    f = run_gpu(sim, trace)
    back = oracle.simulate(cfg, trace.records, trace.offsets, replay=f["lat"], logs=True)
    np.testing.assert_array_equal(back.cycles, f["cycles"])
    return ref, f, err


def test_c1_fp32_teacher_forced_and_free_running():
    w = I.WORKLOADS["c1"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    ref, free, err = teacher_forced_check(w.arch, trace, "fp32", blob)
    # free-running: same CNN on its own trajectory
    check_cpi(abs(free["cycles"].sum() / ref.cycles.sum() - 1.0), "fp32", "c1 free-running")
    agree = (free["lat"] == ref.lat).mean()
    assert agree > 0.99


@pytest.mark.parametrize("lengths", [[0, 1, 5, 33, 130, 7, 64, 0], [1], [257]])
def test_ragged_subtraces_fp32(lengths):
    arch = I.ARCH_SMALL(32)
    trace = I.small_trace(lengths, seed=sum(lengths) + 3)
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=17))
    teacher_forced_check(arch, trace, "fp32", blob)


@pytest.mark.parametrize("rw,strict,graph", [(1, False, True), (3, True, False), (8, True, True)])
def test_retire_rules_fp32(rw, strict, graph):
    arch = I.Arch(window=16, n_conv=1, channels=64, hidden=64)
    trace = I.small_trace([200, 31, 90], seed=5)
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=23))
    teacher_forced_check(arch, trace, "fp32", blob, rw=rw, strict=strict, graph=graph)


def test_c2_arch_fp32_small():
    w = I.WORKLOADS["c2"]
    full = I.make_trace(w, n_subtraces=4)
    offs = np.minimum(full.offsets, 1200)                      # lengths 1000, 200, 0, 0
    trace = I.Trace(full.records[:1200].copy(), offs)
    blob = I.workload_weights(w)
    teacher_forced_check(w.arch, trace, "fp32", blob)


def test_graph_and_direct_launch_identical():
    w = I.WORKLOADS["c1"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    a, _ = make_sim(w.arch, "fp32", blob=blob, graph=True)
    b, _ = make_sim(w.arch, "fp32", blob=blob, graph=False)
    ra, ra2, rb = run_gpu(a, trace), run_gpu(a, trace), run_gpu(b, trace)
    np.testing.assert_array_equal(ra["lat"], rb["lat"])
    np.testing.assert_array_equal(ra["cycles"], rb["cycles"])
    np.testing.assert_array_equal(ra["pre"], ra2["pre"])     # run-to-run bit identical


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_launch_modes_identical(precision):
    """Per-layer kernels with programmatic dependent launch, CUDA graphs and
    plain launches must give bit-identical logs on a workload with compaction
    (uneven lengths)."""
    arch = I.ARCH_SMALL(32)
    trace = I.small_trace([50, 300, 7, 160, 0, 90] * 4, seed=12)
    blob = I.workload_weights(I.Workload("p", arch, 1, 1, seed=12))
    runs = []
    for graph, pdl in ((True, True), (True, False), (False, True), (False, False)):
        sim, _ = make_sim(arch, precision, blob=blob, graph=graph, pdl=pdl, persistent=False)
        runs.append(run_gpu(sim, trace))
    for r in runs[1:]:
        np.testing.assert_array_equal(r["pre"], runs[0]["pre"])
        np.testing.assert_array_equal(r["cycles"], runs[0]["cycles"])


@pytest.mark.parametrize("precision,kernel", [("bf16", "cluster"), ("bf16", "persistent"), ("fp8", "cluster"),
                                              ("fp8", "persistent")])
@pytest.mark.parametrize("case", ["c1", "ragged", "uneven", "c2arch"])
def test_persistent_kernel_teacher_forced(precision, kernel, case):
    """The single-launch kernels against the oracle: the cluster kernel (slots
    owned by clusters of 4 CTAs, state in shared memory, conv pyramid on chip)
    and the grid-wide persistent kernel (padding-extent skipping, pair-major
    layout, compaction inside the kernel).  Integer state bit-exact under
    teacher forcing both ways, latencies within the precision's bound, and
    close to the per-layer path on identical states.  The uneven case has 300
    sub-traces: three clusters, the last one partly empty."""
    if case == "c1":
        w = I.WORKLOADS["c1"]
        arch, trace, blob = w.arch, I.make_trace(w), I.workload_weights(w)
    elif case == "c2arch":
        w = I.WORKLOADS["c2"]
        arch, blob = w.arch, I.workload_weights(w)
        trace = I.small_trace([400, 37, 250, 0, 128], seed=21)
    else:
        arch = I.ARCH_SMALL(32)
        lengths = [0, 1, 5, 33, 130, 7, 64, 0] if case == "ragged" else \
            np.clip(np.rint(np.exp(np.random.default_rng(4).normal(np.log(60), 0.8, 300))), 1, 400).astype(int).tolist()
        trace = I.small_trace(lengths, seed=len(lengths))
        blob = I.workload_weights(I.Workload("u", arch, 1, 1, seed=4))
    cl = kernel == "cluster"
    ref, _, err = teacher_forced_check(arch, trace, precision, blob, persistent=True, cluster=cl, path=kernel)
    lw, _ = make_sim(arch, precision, blob=blob, persistent=False)
    g = run_gpu(lw, trace, replay=ref.lat)
    ps, _ = make_sim(arch, precision, blob=blob, persistent=True, cluster=cl)
    h = run_gpu(ps, trace, replay=ref.lat)
    assert ps.kernel_path == kernel
    np.testing.assert_array_equal(h["cycles"], g["cycles"])
    # two GPU paths on the same state: each is within the row of the oracle, so
    # they are within twice the row of each other
    d = latency_error(h["pre"], g["pre"])
    assert np.median(d) < 1e-3 and d.max() < 2 * LAT_MAX[precision], (np.median(d), d.max())


def test_cluster_kernel_large_batch_four_cta_clusters():
    """2,500 sub-traces of the c2 CNN: 20 clusters, too many for clusters of 8
    to be resident at once, so the kernel runs clusters of 4 CTAs (32 slots
    each); the last cluster is partly empty.  Teacher-forced against the oracle
    with integer state bit-exact."""
    w = I.WORKLOADS["c2"]
    rng = np.random.default_rng(25)
    lengths = rng.integers(1, 24, 2500).tolist()
    trace = I.small_trace(lengths, seed=25)
    teacher_forced_check(w.arch, trace, "bf16", I.workload_weights(w), path="cluster")


def test_cluster_done_before_the_call_ends():
    """Two clusters of the c2 CNN, the first with sub-traces of 12 instructions
    and the second of 150: the first cluster finishes while the call goes on
    (its weight prefetch for a step that never comes must not block it).
    Teacher-forced against the oracle."""
    w = I.WORKLOADS["c2"]
    trace = I.small_trace([12] * 128 + [150] * 128, seed=26)
    teacher_forced_check(w.arch, trace, "bf16", I.workload_weights(w), path="cluster")


def test_long_queues_move_to_the_grid_kernel():
    """Replayed latencies F = 1, E = 200 fill every queue to capacity, so the
    cluster kernel's probe (steps 64-127) sees more than two passes of
    positions a step and the call continues on the grid-wide kernels from the
    same device state (the persistent or the per-layer kernels, whichever its
    timed comparison picks); cycle counts and evictions stay bit-exact.  With
    the path pinned the cluster kernel runs the whole call."""
    w = I.WORKLOADS["c2"]
    trace = I.small_trace([600] * 128, seed=27)
    replay = np.zeros((trace.n_instructions, 2), np.uint8)
    replay[:, 0], replay[:, 1] = 1, 200
    cfg = oracle.Config.of(w.arch)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, replay=replay)
    for auto, paths in ((True, ("persistent", "layerwise")), (False, ("cluster",))):
        sim, _ = make_sim(w.arch, "bf16", blob=I.workload_weights(w), auto_path=auto)
        g = run_gpu(sim, trace, replay=replay)
        assert sim.kernel_path in paths
        np.testing.assert_array_equal(g["cycles"], ref.cycles)
        assert g["stats"].evictions == int(ref.evictions.sum()) > 0


@pytest.mark.parametrize("arch,precision", [(I.ARCH_MID, "fp8"), (I.ARCH_WIDE, "bf16")])
def test_grid_path_choice_keeps_the_state(arch, precision):
    """A long untimed call on the grid-wide path runs 128 steps on the
    persistent kernel, then 64 on it and 64 on the per-layer kernels from the
    same state, timed, and finishes on the faster, so the state passes between
    the two paths at least twice, with compactions on both (sub-traces of
    1,000 and 300 instructions).  Under replayed latencies that fill the queues
    every cycle count and eviction is bit-exact; free-running, the oracle
    replaying the GPU's own latencies reproduces its cycle counts."""
    trace = I.small_trace([1000] * 48 + [300] * 80, seed=29)
    replay = np.zeros((trace.n_instructions, 2), np.uint8)
    replay[:, 0], replay[:, 1] = 1, 200
    cfg = oracle.Config.of(arch)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, replay=replay)
    blob = I.workload_weights(I.Workload("g", arch, 1, 1, seed=29))
    sim, _ = make_sim(arch, precision, blob=blob, auto_path=True)
    assert sim.path_choice == {"persistent_ms": 0.0, "layerwise_ms": 0.0, "steps": 0}
    g = run_gpu(sim, trace, replay=replay)
    assert sim.kernel_path in ("persistent", "layerwise")
    pc = sim.path_choice                     # the comparison that ran: both times measured
    assert pc["steps"] == 32 and pc["persistent_ms"] > 0 and pc["layerwise_ms"] > 0
    np.testing.assert_array_equal(g["cycles"], ref.cycles)
    assert g["stats"].evictions == int(ref.evictions.sum()) > 0
    f = run_gpu(sim, trace)
    back = oracle.simulate(cfg, trace.records, trace.offsets, replay=f["lat"])
    np.testing.assert_array_equal(back.cycles, f["cycles"])


def test_single_long_subtrace_free_running_fp32():
    """One sub-trace of 3,000 instructions (no splitting, B = 1: the reference
    of the sub-trace-length sweep) free-running in FP32 against the FP64
    oracle: CPI within 0.1 %."""
    w = I.WORKLOADS["c2"]
    trace = I.small_trace([3000], seed=28)
    blob = I.workload_weights(w)
    ref = oracle.simulate(oracle.Config.of(w.arch), trace.records, trace.offsets, blob)
    sim, _ = make_sim(w.arch, "fp32", blob=blob)
    g = run_gpu(sim, trace, logs=False)
    check_cpi(abs(g["cycles"].sum() / ref.cycles.sum() - 1.0), "fp32", "3,000-instruction sub-trace")


def test_uneven_lengths_compaction():
    """Log-normal-like uneven lengths exercise the active-set compaction; the
    result must not depend on it (sub-traces are independent, Sec. 3.3)."""
    arch = I.ARCH_SMALL(32)
    rng = np.random.default_rng(4)
    lengths = np.clip(np.rint(np.exp(rng.normal(np.log(60), 0.8, 40))), 1, 400).astype(int).tolist()
    trace = I.small_trace(lengths, seed=44)
    blob = I.workload_weights(I.Workload("u", arch, 1, 1, seed=4))
    teacher_forced_check(arch, trace, "fp32", blob)


def test_cnn_forward_fp32_matches_oracle():
    for arch in (I.ARCH_SMALL(32), I.ARCH_MID, I.ARCH_WIDE):
        blob = I.workload_weights(I.Workload("x", arch, 1, 1, seed=9))
        sim, _ = make_sim(arch, "fp32", blob=blob)
        x = I.random_windows(333, arch, 10)   # 333 windows: several tiles and a ragged tail
        z = sim.cnn_forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
        zr = oracle.cnn_forward(oracle.Config.of(arch), blob, x)
        check(latency_error(oracle.softplus(z), oracle.softplus(zr)), "fp32", f"latencies {arch}")
        check(latency_error(z, zr), "fp32", f"CNN outputs {arch}")


def test_errors_reported():
    arch = I.ARCH_SMALL(32)
    sim = Simnet.for_arch(arch)
    trace = I.small_trace([10, 10], seed=1)
    rec = torch.from_numpy(trace.records.view(np.int32)).cuda()
    off = torch.from_numpy(trace.offsets).cuda()
    with pytest.raises(SimnetError) as e:
        sim.simulate(rec, off)
    assert e.value.status == 5                                  # ESTATE: no weights
    with pytest.raises(SimnetError) as e:
        sim.load_weights(np.zeros(10, np.float32))
    assert e.value.status == 1                                  # EINVAL: wrong blob size
    sim.load_weights(I.workload_weights(I.Workload("x", arch, 1, 1, seed=1)).astype(np.float32))
    bad = torch.tensor([0, 21, 20], dtype=torch.int64, device="cuda")   # offsets decrease
    with pytest.raises(SimnetError) as e:
        sim.simulate(rec, bad)
    assert e.value.status == 1


def test_barrier_timeout_reported_and_context_recovers():
    """Failure detection without a fault: the persistent kernel's grid-barrier
    waits get a 1 us bound (a barrier over 148 CTAs takes longer), so a wait
    gives up, every CTA leaves at a barrier and the call returns ETIMEOUT.  The
    device stays usable: a normal context then reproduces the oracle."""
    w = I.WORKLOADS["c1"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    bad, _ = make_sim(w.arch, "bf16", blob=blob, barrier_limit_us=1, cluster=False)
    with pytest.raises(SimnetError) as e:
        run_gpu(bad, trace)
    assert e.value.status == 4                       # ETIMEOUT
    assert "bound" in str(e.value)
    cfg = oracle.Config.of(w.arch)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, blob, logs=True)
    good, _ = make_sim(w.arch, "bf16", blob=blob, cluster=False)
    g = run_gpu(good, trace, replay=ref.lat)
    np.testing.assert_array_equal(g["cycles"], ref.cycles)
    assert good.kernel_path == "persistent"


def test_cluster_wait_timeout_reported_and_context_recovers():
    """The cluster kernel's waits (on its own pipeline and on the other CTAs
    of the cluster) get a 100 ns bound, so one gives up at once: the CTA
    records a timeout, lets its copies and MMAs land, every CTA leaves at the
    next step boundary, and the call returns ETIMEOUT.  A normal context on the
    same device then reproduces the oracle, and so does the cluster kernel
    given the default bound."""
    w = I.WORKLOADS["c1"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    bad, _ = make_sim(w.arch, "bf16", blob=blob, spin_limit_ns=100)
    with pytest.raises(SimnetError) as e:
        run_gpu(bad, trace)
    assert e.value.status == 4                       # ETIMEOUT
    assert bad.kernel_path == "cluster"
    cfg = oracle.Config.of(w.arch)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, blob, logs=True)
    good, _ = make_sim(w.arch, "bf16", blob=blob)
    g = run_gpu(good, trace, replay=ref.lat)
    assert good.kernel_path == "cluster"
    np.testing.assert_array_equal(g["cycles"], ref.cycles)

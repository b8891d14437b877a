"""The autotuner (simnet_autotune) on the two single-launch kernels.

For a batch size it times launch shapes one knob after another on a
synthetic trace and keeps the fastest: the cluster kernel's cluster size,
weight-stage size and stage count; the persistent kernel's per-phase tile
widths and pipeline stages.  A tuned context must
* report its choice for that batch size (simnet_autotune_plan);
* give the same simulation: under replayed latencies every cycle count is
  bit-identical to an untuned context's, and the predicted latencies agree to
  FP32 rounding (only the split of FC1's FC2 partial sums can move);
* be no slower than the untuned context on a workload of that batch size
  (best of three calls each, 5 % allowance for timing noise).
"""
import numpy as np
import pytest
import torch

from paper_2105_05821_b300 import inputs as I

from gpu_util import latency_error, make_sim, to_dev

pytestmark = pytest.mark.gpu


def best_ms(sim, rec, off, n=3):
    sim.simulate(rec, off, stats=False)
    return min(sim.simulate(rec, off).ms_total for _ in range(n))


@pytest.mark.parametrize("arch,precision,path", [(I.ARCH_MID, "bf16", "cluster"),
                                                  (I.ARCH_MID, "fp8", "persistent"),
                                                  (I.ARCH_WIDE, "bf16", "persistent")])
def test_tuned_plan_same_results_no_slower(arch, precision, path):
    B = 512
    blob = I.workload_weights(I.Workload("a", arch, 1, 1, seed=31))
    trace = I.small_trace([300] * B, seed=31)
    rec, off = to_dev(trace)
    replay = np.stack([np.random.default_rng(1).integers(0, 3, trace.n_instructions),
                       np.random.default_rng(2).integers(0, 30, trace.n_instructions)], 1).astype(np.uint8)
    rp = torch.from_numpy(replay).cuda()
    kw = {} if path == "cluster" else {"cluster": False}
    base, _ = make_sim(arch, precision, blob=blob, **kw)
    tuned, _ = make_sim(arch, precision, blob=blob, **kw)
    widths = tuned.autotune(B, steps=64)
    plan = tuned.autotune_plan()
    print(f"\n{arch} {precision}: {plan}")
    assert plan["batch"] == B and plan["path"] == path
    if path == "cluster":
        assert plan["cluster_size"] in (4, 8) and plan["cluster_stage_bytes"] in (16384, 32768)
        assert plan["cluster_stages"] >= 2
    else:
        assert plan["tile_widths"] == widths[:arch.n_conv + 1] and 2 <= plan["persist_stages"] <= 6
    outs = []
    for sim in (base, tuned):
        N = trace.n_instructions
        pre = torch.full((N, 2), float("nan"), device="cuda")
        sim.simulate(rec, off, pre_log=pre, replay=rp)
        assert sim.kernel_path == path
        outs.append((sim.cycles.cpu().numpy(), pre.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert latency_error(outs[1][1], outs[0][1]).max() <= 1e-4
    t_base, t_tuned = best_ms(base, rec, off), best_ms(tuned, rec, off)
    print(f"untuned {t_base:.3f} ms, tuned {t_tuned:.3f} ms")
    assert t_tuned <= 1.05 * t_base

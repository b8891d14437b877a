"""GPU parity of the tcgen05 tensor-core path (BF16) against the FP64 oracle.

The integer state stays bit-exact under teacher forcing in every precision.
Predicted latencies carry the BF16 rounding of features, weights and
activations (FP32 accumulation); the bounds asserted are the BF16 row of
tests/tolerances.py.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

import oracle
from paper_2105_05821_b300 import inputs as I

from gpu_util import latency_error, make_sim, run_gpu
from test_gpu_sim import teacher_forced_check
from tolerances import check, check_cpi

pytestmark = pytest.mark.gpu


def torch_bf16_reference(arch, blob, x):
    """Plain PyTorch CNN with the kernel's rounding points: BF16 features,
    weights and inter-layer activations, FP32 accumulation, bias and FC2."""
    ws = {k: torch.tensor(v, dtype=torch.float32) for k, v in I.unflatten_weights(arch, blob)}
    q = lambda t: t.to(torch.bfloat16).to(torch.float32)  # noqa: E731
    h = q(torch.tensor(x, dtype=torch.float32)).permute(0, 2, 1)
    for k in range(arch.n_conv):
        h = q(torch.relu(Fn.conv1d(h, q(ws[f"conv{k + 1}.weight"]), ws[f"conv{k + 1}.bias"], stride=2)))
    h = torch.relu(Fn.linear(h.reshape(h.shape[0], -1), q(ws["fc1.weight"]), ws["fc1.bias"]))
    return Fn.linear(h, ws["fc2.weight"], ws["fc2.bias"]).numpy()


def real_windows(arch, seed, n_sub=3, length=120):
    """Feature matrices the simulator really builds: the oracle's per-step
    inputs on a short synthetic trace."""
    trace = I.small_trace([length] * n_sub, seed=seed)
    blob = I.workload_weights(I.Workload("x", arch, 1, 1, seed=9))
    r = oracle.simulate(oracle.Config.of(arch), trace.records, trace.offsets, blob, features=True)
    return r.feat, blob


@pytest.mark.parametrize("arch", [I.ARCH_SMALL(32), I.ARCH_MID, I.ARCH_WIDE, I.ARCH_SMALL(96)])
def test_cnn_forward_bf16(arch):
    """The tcgen05 GEMM chain against a PyTorch CPU reference with the same BF16
    rounding points (tight), and its distance to the FP64 oracle (reported)."""
    x, blob = real_windows(arch, seed=arch.window + arch.n_conv)
    sim, _ = make_sim(arch, "bf16", blob=blob)
    z = sim.cnn_forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    ze = torch_bf16_reference(arch, blob, x)
    d = np.abs(z - ze) / (np.abs(ze) + 1.0)
    zr = oracle.cnn_forward(oracle.Config.of(arch), blob, x)
    print(f"\nbf16 cnn {arch}: vs bf16 reference median {np.median(d):.2e} p99 {np.percentile(d, 99):.2e} "
          f"max {d.max():.2e}")
    # same rounding points, different FP32 summation order inside the tensor core:
    # an occasional BF16 rounding flip of one activation propagates to the output
    assert np.median(d) <= 1e-4 and np.percentile(d, 99) <= 5e-3 and d.max() <= 5e-2
    check(latency_error(oracle.softplus(z), oracle.softplus(zr)), "bf16", f"latencies {arch}")
    check(latency_error(z, zr), "bf16", f"CNN outputs {arch}")


def test_c1_bf16_teacher_forced():
    w = I.WORKLOADS["c1"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    ref, free, err = teacher_forced_check(w.arch, trace, "bf16", blob)
    check_cpi(abs(free["cycles"].sum() / ref.cycles.sum() - 1.0), "bf16", "c1 free-running")


@pytest.mark.parametrize("lengths", [[0, 1, 5, 33, 130, 7, 64, 0], [300] * 40])
def test_ragged_bf16(lengths):
    arch = I.ARCH_SMALL(32)
    trace = I.small_trace(lengths, seed=len(lengths) + 1)
    blob = I.workload_weights(I.Workload("r", arch, 1, 1, seed=17))
    teacher_forced_check(arch, trace, "bf16", blob)


def test_c2_full_size_sampled_bf16():
    """The bench workload at full size (1,024 sub-traces x 1,000), in the bench's
    launch configuration; 8 sampled sub-traces re-simulated by the oracle with
    the GPU's latencies (bit-exact cycles) and their predicted latencies
    checked against the oracle's CNN on the same states."""
    w = I.WORKLOADS["c2"]
    trace = I.make_trace(w)
    blob = I.workload_weights(w)
    sim, _ = make_sim(w.arch, "bf16", blob=blob)
    g = run_gpu(sim, trace)
    ids = [0, 1, 255, 511, 512, 700, 1022, 1023]
    cfg = oracle.Config.of(w.arch)
    ref = oracle.simulate(cfg, trace.records, trace.offsets, blob, subset=ids, replay=g["lat"], logs=True)
    np.testing.assert_array_equal(ref.cycles, g["cycles"][ids])
    sel = np.concatenate([np.arange(trace.offsets[i], trace.offsets[i + 1]) for i in ids])
    check(latency_error(g["pre"][sel], ref.pre[sel]), "bf16", "c2 full size, 8 sampled sub-traces")

"""simnet_cnn_forward_noalloc: the CNN entry point for callers that cannot
allocate device memory while they run (inside an allocator hook, under a
memory budget fixed up front, or in a loop that cannot take cudaMalloc's
synchronisation).  It must give what simnet_cnn_forward gives, and what the
FP64 oracle's CNN gives within the FP32 row of tests/tolerances.py, call after
call, using only the library's fixed scratch array.  Collected last on purpose
(file name)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300 import simnet as S

from gpu_util import latency_error
from tolerances import check

pytestmark = pytest.mark.gpu


def _ctx(arch, precision="fp32"):
    sim = S.Simnet.for_arch(arch, precision=precision)
    blob = I.workload_weights(I.Workload("n", arch, 1, 1, seed=5))
    sim.load_weights(blob.astype(np.float32))
    return sim, blob


def _call_abi(sim, x, z):
    """The new entry point, called through the C ABI directly."""
    return S.lib().simnet_cnn_forward_noalloc(sim._h, ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(z.data_ptr()), x.shape[0],
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_allocating_entry_point_and_oracle_twice():
    assert S.lib().simnet_noalloc_scratch_bytes() == 16 << 20
    # two calls in a row on one context (different sizes), then another context
    cases = [(I.ARCH_SMALL(32), 300, 1), (I.ARCH_SMALL(32), 77, 2), (I.ARCH_MID, 150, 3)]
    sims = {}
    for arch, n, seed in cases:
        sim, blob = sims.setdefault(arch, _ctx(arch))
        xn = I.random_windows(n, arch, seed)
        x = torch.from_numpy(xn.astype(np.float32)).cuda()
        ref = sim.cnn_forward(x).clone()
        z = torch.full((n, 2), float("nan"), device="cuda")
        assert _call_abi(sim, x, z) == 0, S.lib().simnet_last_error(sim._h)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(z).all())
        zc = z.cpu().numpy()
        check(latency_error(zc, ref.cpu().numpy()), "fp32", f"no-alloc vs simnet_cnn_forward, n={n}")
        check(latency_error(zc, oracle.cnn_forward(oracle.Config.of(arch), blob, xn)), "fp32",
              f"no-alloc vs oracle, n={n}")


def test_noalloc_calls_leave_device_memory_unchanged():
    """After a first call (which looks up the scratch array's address and loads
    the kernels), further calls of several sizes change the device's free
    memory by nothing."""
    arch = I.ARCH_SMALL(32)
    sim, _ = _ctx(arch)
    sizes = [300, 1, 77, 512]
    xs = [torch.from_numpy(I.random_windows(n, arch, 40 + n).astype(np.float32)).cuda() for n in sizes]
    zs = [torch.empty((n, 2), device="cuda") for n in sizes]
    for x, z in zip(xs, zs):                      # warm: every size once
        assert _call_abi(sim, x, z) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for x, z in zip(xs, zs):
            assert _call_abi(sim, x, z) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_oversize_and_non_fp32():
    arch = I.ARCH_MID
    sim, _ = _ctx(arch)
    n = 4096                                   # needs far more than the 16 MiB scratch
    x = torch.zeros((n, arch.window, 50), device="cuda")
    z = torch.full((n, 2), 7.0, device="cuda")
    assert _call_abi(sim, x, z) == 1           # EINVAL
    assert b"limit" in S.lib().simnet_last_error(sim._h)
    torch.cuda.synchronize()
    assert bool((z == 7.0).all())              # nothing was written
    b, _ = _ctx(arch, precision="bf16")
    assert _call_abi(b, x[:4], z[:4]) == 6     # EUNSUPPORTED

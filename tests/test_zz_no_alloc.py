"""simnet_cnn_forward_noalloc: the CNN entry point for callers that cannot
allocate device memory (inside an allocator hook, under a memory budget fixed
up front, or in a loop that cannot take cudaMalloc's synchronisation).  It
must give what simnet_cnn_forward gives, call after call, using only the
library's fixed scratch array.  Collected last on purpose (file name)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300 import simnet as S

pytestmark = pytest.mark.gpu

TOL = 1e-3   # the FP32 latency tolerance of the other parity tests, as |a - b| / (|b| + 1)


def _ctx(arch, precision="fp32"):
    sim = S.Simnet.for_arch(arch, precision=precision)
    sim.load_weights(I.workload_weights(I.Workload("n", arch, 1, 1, seed=5)).astype(np.float32))
    return sim


def _call_abi(sim, x, z):
    """The new entry point, called through the C ABI directly."""
    return S.lib().simnet_cnn_forward_noalloc(sim._h, ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(z.data_ptr()), x.shape[0],
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_allocating_entry_point_twice():
    assert S.lib().simnet_noalloc_scratch_bytes() == 16 << 20
    # two calls in a row on one context (different sizes), then another context
    cases = [(I.ARCH_SMALL(32), 300, 1), (I.ARCH_SMALL(32), 77, 2), (I.ARCH_MID, 150, 3)]
    sims = {}
    for arch, n, seed in cases:
        sim = sims.setdefault(arch, _ctx(arch))
        x = torch.from_numpy(I.random_windows(n, arch, seed).astype(np.float32)).cuda()
        ref = sim.cnn_forward(x).clone()
        z = torch.full((n, 2), float("nan"), device="cuda")
        assert _call_abi(sim, x, z) == 0, S.lib().simnet_last_error(sim._h)
        torch.cuda.synchronize()
        d = (z - ref).abs() / (ref.abs() + 1.0)
        assert bool(torch.isfinite(z).all()) and float(d.max()) <= TOL


def test_noalloc_rejects_oversize_and_non_fp32():
    arch = I.ARCH_MID
    sim = _ctx(arch)
    n = 4096                                   # needs far more than the 16 MiB scratch
    x = torch.zeros((n, arch.window, 50), device="cuda")
    z = torch.full((n, 2), 7.0, device="cuda")
    assert _call_abi(sim, x, z) == 1           # EINVAL
    assert b"limit" in S.lib().simnet_last_error(sim._h)
    torch.cuda.synchronize()
    assert bool((z == 7.0).all())              # nothing was written
    b = _ctx(arch, precision="bf16")
    assert _call_abi(b, x[:4], z[:4]) == 6     # EUNSUPPORTED

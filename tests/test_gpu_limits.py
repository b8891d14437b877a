"""Degenerate and limiting inputs of simnet_simulate on every kernel path: a
batch of no sub-traces, sub-traces of no instructions (Eq. 1 with nothing to
fetch and nothing to drain: 0 cycles, as in the oracle), and the longest
sub-trace the library accepts (4,194,303 instructions, so that a 32-bit clock
advancing at most 255 cycles an instruction cannot overflow), one past which
the call is refused before any GPU work."""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import SimnetError

from gpu_util import make_sim, run_gpu

pytestmark = pytest.mark.gpu

ARCH = I.ARCH_SMALL(32)
PATHS = {
    "fp32": ("fp32", {}, "layerwise"),
    "bf16-cluster": ("bf16", {}, "cluster"),
    "bf16-persistent": ("bf16", {"cluster": False}, "persistent"),
    "bf16-layerwise": ("bf16", {"persistent": False}, "layerwise"),
    "fp8-cluster": ("fp8", {}, "cluster"),
}


@pytest.mark.parametrize("path", list(PATHS))
def test_empty_batch_and_empty_subtraces(path):
    precision, kw, _ = PATHS[path]
    sim, blob = make_sim(ARCH, precision, **kw)
    # no sub-traces at all: nothing to do
    rec = torch.zeros(0, dtype=torch.int32, device="cuda")
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = sim.simulate(rec, off)
    assert st.instructions == 0 and st.total_cycles == 0 and st.pending == 0
    # sub-traces of no instructions, alone and beside others
    for lengths in ([0, 0, 0, 0, 0], [0, 3, 0, 1, 0]):
        trace = I.small_trace(lengths, seed=5)
        g = run_gpu(sim, trace)
        ref = oracle.simulate(oracle.Config.of(ARCH), trace.records, trace.offsets, blob, logs=True)
        np.testing.assert_array_equal(g["cycles"], ref.cycles)
        assert (g["cycles"][np.asarray(lengths) == 0] == 0).all()
    sim.close()


def test_subtrace_longer_than_the_limit_is_refused():
    sim, _ = make_sim(ARCH, "bf16")
    n = 4_194_304                                   # one past the limit, after a sub-trace of 2
    rec = torch.zeros(n + 2, dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 2, n + 2], dtype=torch.int64, device="cuda")
    cyc = torch.full((2,), -7, dtype=torch.int64, device="cuda")
    with pytest.raises(SimnetError) as e:
        sim.simulate(rec, off, cycles_out=cyc)
    assert e.value.status == 1                      # EINVAL
    assert "4194303" in str(e.value)
    torch.cuda.synchronize()
    assert (cyc == -7).all()                        # refused before any GPU work
    sim.close()

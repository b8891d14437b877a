"""Sub-trace length against accuracy (Sec. 3.3): a trace cut into sub-traces
that each start from an empty queue and end with their own drain gives a CPI
that drifts from the unsplit trace's as the sub-traces get shorter.

One synthetic trace of 8,192 instructions with the c2 workload's CNN.  The
FP64 oracle simulates it unsplit (the reference) and split into 32 x 256 and
4 x 2,048; the default BF16 GPU path simulates the same splits.  Asserted:
* the GPU split matches the oracle split within the BF16 CPI row of
  tests/tolerances.py (the precision's error, on the same split);
* the split itself costs the oracle less at 2,048 instructions than at 256,
  and at most 1 % at 2,048 (the paper's sub-traces hold thousands of
  instructions for this reason);
* the GPU split against the oracle's unsplit trace stays within the sum of
  the two.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_05821_b300 import inputs as I

from gpu_util import make_sim
from tolerances import CPI, check_cpi

pytestmark = pytest.mark.gpu

N = 8192


@pytest.fixture(scope="module")
def setup():
    w = I.WORKLOADS["c2"]
    records = I.make_records(N, 11)
    blob = I.workload_weights(w)
    cfg = oracle.Config.of(w.arch, retire_width=w.retire_width)
    ref = oracle.simulate(cfg, records, I.equal_offsets(N, 1), blob)
    return w, records, blob, cfg, float(ref.cycles.sum()) / N


def test_split_error_against_the_unsplit_oracle(setup):
    w, records, blob, cfg, cpi_ref = setup
    sim, _ = make_sim(w.arch, "bf16", blob=blob, retire_width=w.retire_width)
    rec = torch.from_numpy(records.view(np.int32).copy()).cuda()
    split_err = {}
    for length in (256, 2048):
        offs = I.equal_offsets(N, N // length)
        o = oracle.simulate(cfg, records, offs, blob)
        cpi_o = float(o.cycles.sum()) / N
        st = sim.simulate(rec, torch.from_numpy(offs).cuda())
        cpi_g = st.total_cycles / N
        assert sim.kernel_path == "cluster"
        check_cpi(abs(cpi_g / cpi_o - 1.0), "bf16", f"GPU vs oracle, {N // length} x {length}")
        split_err[length] = abs(cpi_o / cpi_ref - 1.0)
        print(f"\nsplit {N // length} x {length}: oracle split error {split_err[length]:.2e}, "
              f"GPU vs unsplit oracle {abs(cpi_g / cpi_ref - 1.0):.2e}")
        assert abs(cpi_g / cpi_ref - 1.0) <= split_err[length] + CPI["bf16"]
    assert split_err[2048] < split_err[256]
    assert split_err[2048] <= 0.01

"""The regression head's integer decision on every kernel path, at the
boundaries of its definition: latency = round half to even of softplus(z)
clamped to [0, 255], NaN -> 255 (Sec. 2.3's regression head; the rounding
reading of the design notes).  FC2's weights are zero, so every FC2 output
equals its bias exactly, on the GPU (FP32 FC2 in every precision) as in the
oracle, while the conv and FC1 layers still run their real arithmetic.  The
latencies are compared with the values the rule gives by hand and with the
oracle's, and the cycle counts bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2105_05821_b300 import inputs as I

from gpu_util import make_sim, run_gpu

pytestmark = pytest.mark.gpu

ARCH = I.ARCH_SMALL(32)      # every kernel path takes it

PATHS = {
    "fp32": ("fp32", {}, "layerwise"),
    "bf16-layerwise": ("bf16", {"persistent": False}, "layerwise"),
    "bf16-persistent": ("bf16", {"cluster": False}, "persistent"),
    "bf16-cluster": ("bf16", {}, "cluster"),
    "fp8-layerwise": ("fp8", {"persistent": False}, "layerwise"),
    "fp8-persistent": ("fp8", {"cluster": False}, "persistent"),
    "fp8-cluster": ("fp8", {}, "cluster"),
}

# (fetch bias, execution bias) -> (F, E).  Above 20 softplus is the identity,
# so a bias of k + 0.5 lands exactly on a rounding boundary: half to even.
CASES = {
    "half-to-even": ((22.5, 23.5), (22, 24)),
    "clamp": ((300.0, -50.0), (255, 0)),
    "small": ((0.0, 20.5), (1, 20)),          # softplus(0) = ln 2 -> 1
    "nan": ((float("nan"), 21.49999), (255, 21)),
}


def fc2_bias_only_blob(bf: float, be: float) -> np.ndarray:
    ws = I.he_weights(ARCH, 7)
    ws[-2] = ("fc2.weight", np.zeros_like(ws[-2][1]))
    ws[-1] = ("fc2.bias", np.array([bf, be], dtype=np.float64))
    return I.flatten_weights(ws)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("path", list(PATHS))
def test_rounding_clamp_and_nan_on_every_path(path, case):
    precision, kw, kind = PATHS[path]
    (bf, be), (ef, ee) = CASES[case]
    blob = fc2_bias_only_blob(bf, be)
    trace = I.small_trace([9, 0, 31, 2, 40], seed=13)
    sim, _ = make_sim(ARCH, precision, blob=blob, **kw)
    g = run_gpu(sim, trace)
    assert sim.kernel_path == kind
    assert (g["lat"][:, 0] == ef).all() and (g["lat"][:, 1] == ee).all(), (path, case)
    ref = oracle.simulate(oracle.Config.of(ARCH), trace.records, trace.offsets, blob, logs=True)
    assert (ref.lat[:, 0] == ef).all() and (ref.lat[:, 1] == ee).all()
    np.testing.assert_array_equal(ref.cycles, g["cycles"])
    sim.close()

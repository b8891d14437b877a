"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs."""
import numpy as np
import torch

import oracle
from paper_2105_05821_b300 import inputs as I
from paper_2105_05821_b300.simnet import Simnet


def latency_error(gpu, ref):
    """The paper's prediction error form |f - y| / (y + 1) (Sec. 2.5), on the
    softplus outputs before rounding."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(gpu - ref) / (np.abs(ref) + 1.0)


def to_dev(trace: I.Trace):
    rec = torch.from_numpy(trace.records.view(np.int32).copy()).cuda()
    off = torch.from_numpy(trace.offsets.copy()).cuda()
    return rec, off


def run_gpu(sim: Simnet, trace: I.Trace, replay=None, logs=True):
    rec, off = to_dev(trace)
    N = trace.n_instructions
    NL = sim.n_lat
    lat = torch.zeros((max(N, 1), NL), dtype=torch.uint8, device="cuda") if logs else None
    pre = torch.full((max(N, 1), NL), float("nan"), dtype=torch.float32, device="cuda") if logs else None
    rp = None
    if replay is not None:
        rp = torch.from_numpy(np.ascontiguousarray(replay, dtype=np.uint8)).cuda()
    st = sim.simulate(rec, off, lat_log=lat, pre_log=pre, replay=rp)
    torch.cuda.synchronize()
    out = {"cycles": sim.cycles.cpu().numpy(), "stats": st}
    if logs:
        out["lat"] = lat.cpu().numpy()[:N]
        out["pre"] = pre.cpu().numpy()[:N]
    return out


# Plain PyTorch statements of the training losses (Sec. 2.4; the hybrid head's
# cross-entropy of Sec. 2.3), the references the library's loss kernels are
# checked against.
def mse_softplus(z: torch.Tensor, labels: torch.Tensor) -> torch.Tensor:
    """Mean over all outputs of (softplus(z) - clamp(label, 0, 255))^2."""
    return (torch.nn.functional.softplus(z) - labels.float().clamp(0, 255)).pow(2).mean()


def hybrid_loss(z: torch.Tensor, labels: torch.Tensor) -> torch.Tensor:
    """Hybrid head (Sec. 2.3) loss on z [n, 22]: mean over the 2n latencies of the
    cross-entropy of the ten class logits against class min(label, 9) plus the
    squared error of softplus(regression output) against the label."""
    y = labels.float().clamp(0, 255)
    total = z.new_zeros(())
    for t in range(2):
        cls = y[:, t].clamp(max=9).long()
        ce = torch.nn.functional.cross_entropy(z[:, 11 * t:11 * t + 10], cls, reduction="sum")
        se = (torch.nn.functional.softplus(z[:, 11 * t + 10]) - y[:, t]).pow(2).sum()
        total = total + ce + se
    return total / (2 * z.shape[0])



def make_sim(arch, precision="fp32", blob=None, seed=None, **kw):
    kw.setdefault("auto_path", False)   # a test pins its path unless it tests the choice
    sim = Simnet.for_arch(arch, precision=precision, **kw)
    if blob is None:
        blob = I.workload_weights(I.Workload("x", arch, 1, 1, seed=seed or 1))
    sim.load_weights(blob.astype(np.float32))
    return sim, blob

"""The benchmark stays on one GPU: launched with more than one rank it runs no
GPU work, rank 0 prints one line that says so, and every rank exits 0.  The
CPU reference arm under the same launch runs on rank 0 alone.  Run as
subprocesses with the rank environment set (no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(rank, *extra):
    env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *extra], env=env, cwd=ROOT,
                          capture_output=True, text=True, timeout=300)


def test_more_than_one_rank_runs_no_gpu_work():
    r0, r1 = _bench(0), _bench(1)
    assert r0.returncode == 0 and r1.returncode == 0, (r0.stderr, r1.stderr)
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["n_gpus"] == 2 and "one GPU only" in line["unavailable"]
    assert r1.stdout.strip() == ""


def test_reference_arm_runs_on_rank_zero_only():
    r1 = _bench(1, "--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "c1")
    assert r1.returncode == 0 and r1.stdout.strip() == ""


def test_reference_arm_line_on_one_rank():
    """The reference arm's JSON line (the FP64 oracle timed on the host cores):
    the bench contract's keys, its own value as the CPU baseline, and an
    end-to-end figure with no host-device traffic."""
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "c1"], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "inst/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0 and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "inst/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("c1:")

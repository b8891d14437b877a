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

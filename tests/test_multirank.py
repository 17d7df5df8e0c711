"""The bench's multi-rank host logic on CPU (gloo, world size 2): the step time
is the slowest rank's, the value sums every rank's work over it, and under
torchrun the reference arm runs on rank 0 only (other ranks exit 0 silently).
The GPU path itself needs no collective: every rank runs its own copy of the
independent (obstacle, mode) tasks."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        ms = bench.slowest_rank_ms(1.5 + rank, torch.device("cpu"))   # rank 1 is slower
        out[rank] = ms
    finally:
        dist.destroy_process_group()


def test_slowest_rank_time_and_job_value():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 2.5
    # two ranks, 1e9 flops each, 2.5 ms for the slowest: 2e9 / 2.5e-3 s = 0.8 TFLOP/s
    assert bench.job_value(2, 1e9, 2.5) == pytest.approx(0.8)


def test_single_rank_is_identity():
    assert bench.slowest_rank_ms(3.25, torch.device("cpu")) == 3.25


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""

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


def _shard_rank(rank, port, out):
    """One process of the mode-sharded operator, on CPU: the library's host
    plan splits the (obstacle, mode) tasks; the oracle stands in for the GPU
    solve of the owned modes; the binding's all-reduce assembles them."""
    import numpy as np
    import oracle as O
    import synth
    from paper_1506_05083_gb300 import axi
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        obs = [synth.small_case(seed=7).obstacles[0],
               synth.small_case(seed=11, k=2.0, M=44, N=36, P=20, bc=synth.BC_TRANSMISSION).obstacles[0]]
        specs = [axi.spec_from_obstacle(ob) for ob in obs]
        plan = axi.Plan(specs)
        plan.shard(rank, 2)
        masks = [plan.owned_modes(i) for i in range(len(obs))]
        coefs, fulls = [], []
        for i, ob in enumerate(obs):
            ob = synth.Obstacle(**{**ob.__dict__, "q": specs[i].q})
            coll, src, srcx = O.geometry(ob)
            A, fac = O.factor_operator(ob, coll, src, srcx)
            dirs = synth.plane_wave_directions(3, 70 + i)
            fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
            full = O.solve_modes(ob, fac, fh)
            mine = np.zeros_like(full)
            for idx in range(ob.P):
                n = idx if idx <= ob.P // 2 else ob.P - idx
                if masks[i][n]:
                    mine[:, idx] = full[:, idx]
            c = torch.tensor(mine)
            axi.gather_coefficients(c)
            coefs.append(c.numpy())
            fulls.append(full)
        out[rank] = ([m.tolist() for m in masks], [np.abs(c - f).max() for c, f in zip(coefs, fulls)])
    finally:
        dist.destroy_process_group()


def test_mode_sharding_partition_and_gather():
    """axi_plan_shard over two processes: the owned modes are disjoint and
    cover every (obstacle, mode) task, the QR work is balanced, and the
    gathered coefficients equal the unsharded solution exactly."""
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_shard_rank, args=(port, out), nprocs=2, join=True)
    m0, err0 = out[0]
    m1, err1 = out[1]
    for a, b in zip(m0, m1):
        a, b = list(map(bool, a)), list(map(bool, b))
        assert not any(x and y for x, y in zip(a, b))
        assert all(x or y for x, y in zip(a, b))
    # task costs: 8 rows cols^2 - 8 cols^3 / 3 per distinct mode
    cost = [8 * 40 * 32 ** 2 - 8 * 32 ** 3 / 3, 8 * 88 * 72 ** 2 - 8 * 72 ** 3 / 3]
    loads = [sum(c * sum(map(bool, m)) for c, m in zip(cost, ms)) for ms in (m0, m1)]
    assert abs(loads[0] - loads[1]) <= max(cost)
    assert max(err0) == 0.0 and max(err1) == 0.0

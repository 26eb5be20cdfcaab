"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2)
take distinct batches, time the job as the slowest rank and report the
whole-job throughput; the reference arm's non-zero ranks exit without work."""

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    theta = workloads.theta_box(16, bench.shard_theta_seed(rank))
    local_ms = 10.0 * (rank + 1)
    total = bench.max_over_ranks(local_ms, dist)
    value = bench.whole_job_value(world, 5, 16, total)
    out.put((rank, theta, total, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, th0, t0, v0), (_, th1, t1, v1) = res
    assert not np.array_equal(th0, th1)          # each rank its own points
    assert t0 == t1 == 20.0                      # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 5 * 16 / 0.020)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_value(1, 10, 65536, 20.0) == pytest.approx(10 * 65536 / 0.02)

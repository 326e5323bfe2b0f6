"""The benchmark's multi-rank path on CPU (gloo, world size 2): each rank
times its own replica; the job's time is the slowest rank's and the value is
the units of all ranks over that time. The reference arm runs on rank 0
only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, local_ms, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.max_over_ranks(local_ms[rank], dist)
    v = bench.job_value(world, 1000, 5, m / 1e3)
    dist.barrier()
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local_ms = [10.0, 25.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, m, v in out:
        assert m == 25.0
        assert v == pytest.approx(2 * 1000 * 5 / 0.025)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 10, 2, 4.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        size, warmup, steps, gpus = 4, 1, 1, 2
    # a non-zero rank returns at once, without touching the oracle
    assert bench.run_reference(A(), 1, 2) == 0

"""The multi-GPU form is independent replicas (one problem per rank, no
data-path collective): the bench's barrier, max-over-ranks timing and
whole-job aggregation, run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = bench.max_over_ranks(world, 10.0 + 5.0 * rank)  # rank 1 is the slow one
    v = bench.whole_job_value(world, 2e9, 20, t)
    bench.barrier(world)
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in got:
        assert t == 15.0  # every rank sees the slowest time
        assert abs(v - 2 * 2e9 * 20 / 15e-3 / 1e9) < 1e-9  # both replicas' bytes / max time


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 3.0) == 3.0
    assert abs(bench.whole_job_value(1, 1e9, 10, 2.0) - 5000.0) < 1e-9

"""The N > 1 path of bench.py (replicas, no data-path collective): the max over ranks of the
timed region and the whole-job throughput, run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 1000.0 * (rank + 1)  # rank 1 is the slow one
    mx = bench.max_over_ranks(my_ms, world, "cpu")
    val = bench.throughput(steps=5, solves_per_step=3, world=world, max_ms=mx)
    q.put((rank, mx, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, val in out:
        assert mx == 2000.0                    # every rank sees the slowest rank's time
        assert abs(val - 5 * 3 * 2 / 2.0) < 1e-12  # 30 solves over 2 s


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(123.0, 1) == 123.0
    assert bench.throughput(4, 3, 1, 2000.0) == 6.0

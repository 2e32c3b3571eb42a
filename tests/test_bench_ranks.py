"""The bench's multi-rank path on the CPU: two gloo ranks (127.0.0.1), each an independent
replica; the only exchange is the maximum of the per-rank timings, and the whole-job rate
counts every rank's units over the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_info()
    t = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * (rank + 1)], "cpu")
    rate = bench.whole_job_rate(ws, 20, t[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ws, r, local, t, rate))


def test_two_gloo_ranks_take_the_max_and_count_all_units():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, t, rate in out:
        assert (ws, r, local) == (2, rank, rank)
        assert t == [2.0, 10.0, 1.0]              # element-wise maximum over the two ranks
        assert rate == pytest.approx(2 * 20 / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0

"""The N > 1 path of bench.py on CPU: two gloo ranks run the same timing
aggregation as the GPU ranks (max over ranks, whole-job rate) -- the replicas
exchange nothing else."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [10.0 + rank * 5.0, 20.0 - rank * 3.0]   # rank 1 slower on the step, faster end to end
    got = bench.max_over_ranks(mine, dist, "cpu")
    rate = bench.whole_job_rate(633, world, got[0])
    dist.barrier()
    q.put((rank, got, rate))
    dist.destroy_process_group()


def test_two_ranks_agree_on_max_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [15.0, 20.0]
        assert abs(rate - 633 * 2 / 0.015) < 1e-6


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
    assert bench.whole_job_rate(633, 1, 125.0) == pytest.approx(5064.0)

"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
replica (no data-path collective), the timing reduced to the slowest rank and
the rate summed over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws)     # rank 1 is the slow one
    rate = bench.whole_job_rate(3, 4, ws, ms)
    dist.barrier()
    q.put((r, ws, local, ms, rate))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    for _, _, _, ms, rate in out:
        assert ms == 15.0
        assert abs(rate - 2 * 3 * 4 / 0.015) < 1e-9

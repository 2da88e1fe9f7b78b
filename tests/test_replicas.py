"""Two-rank (gloo, CPU) check of the replica aggregation used by bench.py --gpus N: every
rank sees the maximum time over ranks, and throughput counts the work of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_2509_06433_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w = replicas.rank_and_world()
    replicas.barrier()
    m = replicas.max_over_ranks(1.5 + rank)  # rank 1 is the slow one
    q.put((r, w, m, replicas.replica_throughput(100, w, m)))
    dist.destroy_process_group()


def test_two_rank_max_time_and_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == pytest.approx(2.5) for o in out)
    assert all(o[3] == pytest.approx(200 / 2.5) for o in out)


def test_single_process_is_identity():
    from paper_2509_06433_gb300 import replicas
    assert replicas.max_over_ranks(3.25) == 3.25
    assert replicas.replica_throughput(10, 1, 2.0) == 5.0

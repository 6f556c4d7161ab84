"""N>1 host logic on CPU with gloo (world size 2): row partitions are disjoint
and contiguous, the step time is the max over ranks, the job rate counts every
rank's rows."""
import os
import socket

import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2008_03260_b300.multi import job_throughput, max_over_ranks, rank_rows
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    row0, n = rank_rows(rank, world, 1000)
    t = max_over_ranks([0.5 + rank, 2.0 - rank])          # per-rank (insert, query) seconds
    rate = job_throughput(n, world, t[0])
    dist.barrier()
    q.put((rank, row0, n, t, rate))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, n0, t0, v0), (r1, a1, n1, t1, v1) = out
    assert (a0, n0, a1, n1) == (0, 1000, 1000, 1000)      # disjoint, contiguous partitions
    assert t0 == t1 == [1.5, 2.0]                         # max over ranks, element-wise
    assert v0 == v1 == 2000 / 1.5

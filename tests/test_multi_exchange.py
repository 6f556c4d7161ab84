"""One logical index over W ranks (Sec. 3 partitions, Algorithm 2's merge
across machines as one candidate exchange): world size 2 over gloo on CPU.
Each rank's local steps are computed here by the oracle (test side); the
exchange logic and collectives are the product's (paper_2008_03260_b300.multi).
The answer must equal, bit for bit, the oracle's one-index answer whose two
shards are the two ranks' partitions."""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp

import datagen
import oracle

N, K, L, B, R, D, W_CM, SEED = 6000, 4, 16, 9, 16, 4, 1024, 7


class OraclePart:
    """One rank's three local steps, computed by the oracle on its partition."""

    def __init__(self, rank: int, world: int, offs, cols):
        from paper_2008_03260_b300.multi import partition
        lo, n = partition(rank, world, N)
        self.ix = oracle.Index(K=K, L=L, log2_buckets=B, reservoir=R, cm_rows=D, cm_width=W_CM, shards=1,
                               seed=SEED, capacity=N)
        self.ix.set_next_id(lo)
        o = offs[lo:lo + n + 1]
        self.ix.insert(o - o[0], cols[int(o[0]):int(o[-1])])
        self.sc = oracle.derive_seeds(SEED, L, D)["sc"]
        self.m = L * R
        self.sketch = {}

    def empty(self, k):
        return torch.zeros((0, k), dtype=torch.int32), torch.zeros((0, k), dtype=torch.int32)

    def _detail(self, offs, cols, q):
        return self.ix.query_detail(cols[int(offs[q]):int(offs[q + 1])], 1)

    def candidates(self, offs, cols):
        nq = len(offs) - 1
        cnt = torch.zeros(nq, dtype=torch.int32)
        ids = torch.full((nq, self.m), -1, dtype=torch.int32)
        for q in range(nq):
            u = self._detail(offs, cols, q)["U"]
            cnt[q] = len(u)
            ids[q, :len(u)] = torch.from_numpy(u.astype(np.int32))
        return cnt, ids

    def cells(self, offs, cols, ids, cnt):
        world, nq, m = ids.shape
        out = torch.zeros((world, nq, m, D), dtype=torch.int32)
        for q in range(nq):
            cm = self._detail(offs, cols, q)["cm"]
            for w in range(world):
                for j in range(int(cnt[w, q])):
                    x = int(ids[w, q, j])
                    for r in range(D):
                        out[w, q, j, r] = int(cm[r, oracle.cm_cell(x, int(self.sc[r]), W_CM)])
        return out

    def rank(self, ids, cnt, cells, k):
        world, nq, m = ids.shape
        out_i = torch.full((nq, k), -1, dtype=torch.int32)
        out_s = torch.zeros((nq, k), dtype=torch.int32)
        for q in range(nq):
            cand = [(int(cells[w, q, j].min()), int(ids[w, q, j])) for w in range(world) for j in range(int(cnt[w, q]))]
            cand.sort(key=lambda t: (-t[0], t[1]))
            for i, (e, x) in enumerate(cand[:k]):
                out_i[q, i], out_s[q, i] = x, e
        return out_i, out_s


def _inputs():
    g = datagen.Generator()
    offs, cols = g.rows(SEED, 0, N)
    qo, qc, _ = g.queries(SEED, 8, 120, N, planted_frac=0.5, p_perturb=0.2)
    return offs, cols, qo, qc


def _one_index_answer(offs, cols, qo, qc, k):
    ix = oracle.Index(K=K, L=L, log2_buckets=B, reservoir=R, cm_rows=D, cm_width=W_CM, shards=2, seed=SEED,
                      capacity=N)
    ix.insert(offs, cols)
    return ix.query(qo, qc, k)


def test_partitions_are_the_shards_of_one_index():
    from paper_2008_03260_b300.multi import partition
    assert [partition(r, 3, 10) for r in range(3)] == [(0, 4), (4, 3), (7, 3)]
    for n, w in ((6000, 2), (7, 4), (1, 1)):
        parts = [partition(r, w, n) for r in range(w)]
        assert parts[0][0] == 0 and sum(p[1] for p in parts) == n
        # shard(id) = floor(id * w / n) of every id in partition r is r
        for r, (lo, cnt) in enumerate(parts):
            assert all((i * w) // n == r for i in range(lo, lo + cnt))


def test_loopback_exchange_equals_one_index():
    from paper_2008_03260_b300.multi import exchange_query_loopback
    offs, cols, qo, qc = _inputs()
    parts = [OraclePart(r, 2, offs, cols) for r in range(2)]
    ids, sc = exchange_query_loopback(parts, qo, qc, 10, chunk=50)
    want_ids, want_sc = _one_index_answer(offs, cols, qo, qc, 10)
    assert np.array_equal(ids.numpy(), want_ids)
    assert np.array_equal(sc.numpy().astype(np.uint32), want_sc)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2008_03260_b300.multi import TorchComm, exchange_query
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    offs, cols, qo, qc = _inputs()
    part = OraclePart(rank, world, offs, cols)
    ids, sc = exchange_query(part, TorchComm(), qo, qc, 10, chunk=64)
    q.put((rank, ids.numpy(), sc.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo_exchange_equals_one_index():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted((q.get(timeout=300) for _ in ps), key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    offs, cols, qo, qc = _inputs()
    want_ids, want_sc = _one_index_answer(offs, cols, qo, qc, 10)
    for _, ids, sc in out:               # every rank holds the whole answer
        assert np.array_equal(ids, want_ids)
        assert np.array_equal(sc.astype(np.uint32), want_sc)

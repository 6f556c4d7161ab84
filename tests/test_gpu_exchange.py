"""The candidate exchange's device steps (one GPU, the ranks held by one
process): two partition indexes answer a query batch as one logical index,
bit-exactly equal to the oracle's two-shard index and to the one-GPU sharded
index (slash_query with shards = 2)."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    a = a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("world,R,B,k", [(2, 16, 9, 10), (3, 32, 7, 25), (2, 128, 12, 100)])
def test_exchange_equals_one_sharded_index(world, R, B, k):
    import paper_2008_03260_b300 as s
    from paper_2008_03260_b300.multi import GpuPart, exchange_query_loopback, partition
    g = datagen.Generator()
    n = 9000
    offs, cols = g.rows(41, 0, n)
    qo, qc, _ = g.queries(41, 42, 300, n, planted_frac=0.5, p_perturb=0.2)
    base = dict(K=4, L=16, log2_buckets=B, reservoir=R, cm_rows=4, cm_width=2048, seed=41, capacity=n)
    parts, ixs = [], []
    for r in range(world):
        lo, cnt = partition(r, world, n)
        ix = s.Index(s.Params(**base, shards=1))
        ix.set_next_id(lo)
        o = offs[lo:lo + cnt + 1]
        assert ix.insert(_dev(o - o[0]), _dev(cols[int(o[0]):int(o[-1])])) == lo
        ixs.append(ix)
        parts.append(GpuPart(ix))
    d_qo, d_qc = _dev(qo), _dev(qc)
    ids, sc = exchange_query_loopback(parts, d_qo, d_qc, k, chunk=128)
    torch.cuda.synchronize()
    for ix in ixs:
        ix.sync()
        ix.close()
    oix = oracle.Index(K=4, L=16, log2_buckets=B, reservoir=R, cm_rows=4, cm_width=2048, shards=world, seed=41,
                       capacity=n)
    oix.insert(offs, cols)
    want_ids, want_sc = oix.query(qo, qc, k)
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), want_sc)
    with s.Index(s.Params(**base, shards=world)) as one:
        one.insert(_dev(offs), _dev(cols))
        i1, s1 = one.query(d_qo, d_qc, k)
        one.sync()
    assert np.array_equal(i1.cpu().numpy(), want_ids) and np.array_equal(s1.cpu().numpy().view(np.uint32), want_sc)

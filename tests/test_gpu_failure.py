"""Failure handling on the GPU without a GPU fault: an allocation failure made
on the host (the library's test hook) and a bounded device wait that runs out
(a copy wait told to expect bytes that never come).  Both leave the index and
the device usable, and the results afterwards still equal the oracle's."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    a = a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle(p, offs, cols):
    ix = oracle.Index(K=p.K, L=p.L, log2_buckets=p.log2_buckets, reservoir=p.reservoir, cm_rows=p.cm_rows,
                      cm_width=p.cm_width, shards=p.shards, seed=p.seed, capacity=p.capacity)
    ix.insert(offs, cols)
    return ix


def test_insert_allocation_failure_leaves_the_index_unchanged():
    import paper_2008_03260_b300 as s
    g = datagen.Generator()
    n = 12_000
    offs, cols = g.rows(31, 0, n)
    p = s.Params(K=4, L=16, log2_buckets=10, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=31)
    d_cols = _dev(cols)
    with s.Index(p) as ix:
        ix.insert(_dev(offs[:1001]), d_cols)       # workspace for 1000 rows
        ix.sync()
        slots0, fill0 = ix.export()
        s.slash_debug_fail_alloc(ix.h, 1)           # the next workspace allocation fails
        with pytest.raises(s.SlashError) as e:
            ix.insert(_dev(offs[1000:]), d_cols)    # needs a larger workspace
        assert e.value.code == s.SLASH_ENOMEM
        assert ix.size == 1000
        slots1, fill1 = ix.export()
        assert np.array_equal(slots0, slots1) and np.array_equal(fill0, fill1)
        assert ix.insert(_dev(offs[1000:]), d_cols) == 1000   # the same call succeeds afterwards
        ix.sync()
        slots, fill = ix.export()
        # plain queries need a workspace too
        qo, qc, _ = g.queries(31, 32, 300, n)
        s.slash_debug_fail_alloc(ix.h, 1)
        with pytest.raises(s.SlashError) as e:
            ix.query(_dev(qo), _dev(qc), 10, mode="plain")
        assert e.value.code == s.SLASH_ENOMEM
        ids, sc = ix.query(_dev(qo), _dev(qc), 10, mode="plain")
        ix.sync()
    oix = _oracle(p, offs, cols)
    ws, wf = oix.export()
    assert np.array_equal(fill, wf) and np.array_equal(slots, ws)
    want_ids, want_sc = oix.query(qo, qc, 10)
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), want_sc)


def test_bounded_copy_wait_times_out_and_reports():
    import paper_2008_03260_b300 as s
    g = datagen.Generator()
    n = 5000
    offs, cols = g.rows(33, 0, n)
    qo, qc, _ = g.queries(33, 34, 200, n)
    p = s.Params(K=4, L=16, log2_buckets=12, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=33)
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        ix.sync()
        s.slash_debug_stall_copies(ix.h, True)
        ix.query(_dev(qo), _dev(qc), 10, mode="fused")   # every copy wait gives up after its limit
        assert s.slash_sync(ix.h) == s.SLASH_ETIMEOUT
        assert s.slash_sync(ix.h) == s.SLASH_OK           # reported once, then cleared
        s.slash_debug_stall_copies(ix.h, False)
        ids, sc = ix.query(_dev(qo), _dev(qc), 10, mode="fused")
        ix.sync()
    want_ids, want_sc = _oracle(p, offs, cols).query(qo, qc, 10)
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), want_sc)

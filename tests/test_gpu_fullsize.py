"""Full-size parity: the `criteo` workload (50M rows, K=6, L=64, 2^18 buckets,
R=128) inserted in one call and queried with the index's default schedule, as
the benchmark runs it.  The oracle cannot build the whole index quickly, so it
builds only the sampled buckets -- every bucket of 200 sampled queries (chosen
by the oracle's own hashes) plus 2000 random buckets -- from all 50M rows, and
the GPU's copies of those buckets and its answers to those queries must match
bit for bit."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from datagen.workloads import CRITEO as w

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _dev(a):
    return torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32)).cuda()


def test_criteo_full_size_sampled_parity():
    import paper_2008_03260_b300 as s
    g = datagen.Generator()
    offs, cols = g.rows(w.seed, 0, w.n_rows)
    qo, qc, _ = g.queries(w.seed, w.qseed, 200, w.n_rows, **w.query_kwargs())
    p = s.Params(**w.params())
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        ids, sc = ix.query(_dev(qo), _dev(qc), w.topk)
        ix.sync()
        _, qbk = oracle.hash_rows(w.K, w.L, w.log2_buckets, w.seed, w.cm_rows, qo, qc, want_codes=False)
        rng = np.random.default_rng(5)
        rt = np.concatenate([np.tile(np.arange(w.L), len(qo) - 1), rng.integers(0, w.L, 2000)]).astype(np.uint32)
        rb = np.concatenate([qbk.ravel(), rng.integers(0, 1 << w.log2_buckets, 2000)]).astype(np.uint32)
        gslots, gfill = ix.buckets(np.zeros_like(rt), rt, rb)
        gids, gsc = ids.cpu().numpy(), sc.cpu().numpy().view(np.uint32)
    oix = oracle.Index(K=w.K, L=w.L, log2_buckets=w.log2_buckets, reservoir=w.reservoir, cm_rows=w.cm_rows,
                       cm_width=w.cm_width, seed=w.seed, capacity=w.n_rows, partial=(rt, rb))
    oix.insert(offs, cols, threads=datagen.default_threads())
    for i in range(len(rt)):
        want, wf = oix.bucket(int(rt[i]), int(rb[i]))
        assert gfill[i] == wf and np.array_equal(gslots[i], want), (int(rt[i]), int(rb[i]))
    assert gfill.max() == w.reservoir  # the sample includes full (sub-sampled) buckets
    want_ids, want_sc = oix.query(qo, qc, w.topk)
    assert np.array_equal(gids, want_ids)
    assert np.array_equal(gsc, want_sc)


def test_topkapi_full_size_sampled_parity():
    """The `topkapi` workload (50M rows, 4x32 sketches, 2^18 per table) as the
    benchmark runs it: the sketches of 200 queries plus 2000 random ones, and
    the 200 queries' answers, against an oracle that keeps only those sketches
    (its cell updates run in id order over all 50M rows)."""
    import paper_2008_03260_b300 as s
    from datagen.workloads import TOPKAPI as tw
    W, C = tw.extra["tk_rows"], tw.extra["tk_cells"]
    g = datagen.Generator()
    offs, cols = g.rows(tw.seed, 0, tw.n_rows)
    qo, qc, _ = g.queries(tw.seed, tw.qseed, 200, tw.n_rows, **tw.query_kwargs())
    p = s.TkParams(dim=tw.dim, K=tw.K, L=tw.L, log2_buckets=tw.log2_buckets, rows=W, cells=C,
                   seed=tw.seed, capacity=tw.n_rows)
    with s.TkIndex(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        ids, sc = ix.query(_dev(qo), _dev(qc), tw.topk)
        ix.sync()
        _, qbk = oracle.hash_rows(tw.K, tw.L, tw.log2_buckets, tw.seed, W, qo, qc, want_codes=False)
        rng = np.random.default_rng(6)
        rt = np.concatenate([np.tile(np.arange(tw.L), len(qo) - 1), rng.integers(0, tw.L, 2000)]).astype(np.uint32)
        rb = np.concatenate([qbk.ravel(), rng.integers(0, 1 << tw.log2_buckets, 2000)]).astype(np.uint32)
        gcells = ix.buckets(np.zeros_like(rt), rt, rb)
        gids, gsc = ids.cpu().numpy(), sc.cpu().numpy().view(np.uint32)
    oix = oracle.TkIndex(K=tw.K, L=tw.L, log2_buckets=tw.log2_buckets, rows=W, cells=C, seed=tw.seed,
                         capacity=tw.n_rows, partial=(rt, rb))
    oix.insert(offs, cols, threads=datagen.default_threads())
    for i in range(len(rt)):
        cells = oix.bucket(int(rt[i]), int(rb[i]))
        want = np.where(cells[..., 1] > 0, cells[..., 0] + 1, 0).astype(np.uint32)
        assert np.array_equal(gcells[i], want), (int(rt[i]), int(rb[i]))
    assert (gcells > 0).mean() > 0.5  # the sample's sketches are mostly occupied
    want_ids, want_sc = oix.query(qo, qc, tw.topk)
    assert np.array_equal(gids, want_ids)
    assert np.array_equal(gsc, want_sc)


def test_stream_at_scale_sampled_parity():
    """The `stream` shape (K=8, L=32, 2^20 buckets per table, R=256, top-100)
    with 64M rows generated on the device in 16M-row chunks and never stored:
    the buckets of 200 queries plus 2000 random buckets, and the 200 answers,
    against an oracle that keeps only those buckets and takes all 64M rows from
    the host generator (64M rows: the largest stream whose host-side oracle
    finishes within a test's time on the machine's cores)."""
    import paper_2008_03260_b300 as s
    from datagen.workloads import STREAM as sw
    n, chunk = 64 << 20, sw.extra["chunk_rows"]
    g = datagen.Generator()
    dg = datagen.DeviceRows(g)
    p = s.Params(**sw.params(capacity=n))
    qo, qc, _ = g.queries(sw.seed, sw.qseed, 200, n, **sw.query_kwargs())
    with s.Index(p) as ix:
        for r0 in range(0, n, chunk):
            o, c = dg.rows(sw.seed, r0, min(chunk, n - r0), lo=sw.nnz_lo, hi=sw.nnz_hi)
            ix.insert(o, c)
            del o, c
        ids, sc = ix.query(_dev(qo), _dev(qc), sw.topk)
        ix.sync()
        _, qbk = oracle.hash_rows(sw.K, sw.L, sw.log2_buckets, sw.seed, sw.cm_rows, qo, qc, want_codes=False)
        rng = np.random.default_rng(6)
        rt = np.concatenate([np.tile(np.arange(sw.L), len(qo) - 1), rng.integers(0, sw.L, 2000)]).astype(np.uint32)
        rb = np.concatenate([qbk.ravel(), rng.integers(0, 1 << sw.log2_buckets, 2000)]).astype(np.uint32)
        gslots, gfill = ix.buckets(np.zeros_like(rt), rt, rb)
        gids, gsc = ids.cpu().numpy(), sc.cpu().numpy().view(np.uint32)
    oix = oracle.Index(K=sw.K, L=sw.L, log2_buckets=sw.log2_buckets, reservoir=sw.reservoir, cm_rows=sw.cm_rows,
                       cm_width=sw.cm_width, seed=sw.seed, capacity=n, partial=(rt, rb))
    for r0 in range(0, n, chunk):
        o, c = g.rows(sw.seed, r0, min(chunk, n - r0), lo=sw.nnz_lo, hi=sw.nnz_hi)
        assert oix.insert(o - o[0], c, threads=datagen.default_threads()) == r0
        del o, c
    for i in range(len(rt)):
        want, wf = oix.bucket(int(rt[i]), int(rb[i]))
        assert gfill[i] == wf and np.array_equal(gslots[i], want), (int(rt[i]), int(rb[i]))
    assert gfill.sum() > 0
    want_ids, want_sc = oix.query(qo, qc, sw.topk)
    assert np.array_equal(gids, want_ids)
    assert np.array_equal(gsc, want_sc)

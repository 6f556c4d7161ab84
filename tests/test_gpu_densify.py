"""GPU parity of optimal densification (SLASH_DENSIFY_OPTIMAL) against the
oracle: codes, addresses, bucket arrays, query results and sketch buckets."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from test_gpu_parity import _dev, _host_u32, _with_edges

pytestmark = pytest.mark.gpu


def _s():
    import paper_2008_03260_b300 as s
    return s


@pytest.mark.parametrize("K,L,B", [(4, 16, 16), (6, 64, 18), (3, 7, 5), (1, 1, 1), (16, 64, 20), (2, 5, 9)])
def test_optimal_codes_and_addresses(K, L, B):
    s = _s()
    g = datagen.Generator()
    # lognormal query rows reach down to 1 feature: long probe sequences
    qo, qc, _ = g.queries(3, 4, 2000, 1000, planted_frac=0.0)
    offs, cols = _with_edges(qo, qc, 1 << 20)
    p = s.Params(K=K, L=L, log2_buckets=B, reservoir=4, cm_rows=2, cm_width=64, capacity=10_000, seed=11,
                 densify=s.SLASH_DENSIFY_OPTIMAL)
    with s.Index(p) as ix:
        codes, bk = ix.debug_hash(_dev(offs), _dev(cols))
        torch.cuda.synchronize()
        want_codes, want_bk = oracle.hash_rows(K, L, B, 11, 2, offs, cols, densify=1)
        assert np.array_equal(_host_u32(codes), want_codes)
        assert np.array_equal(_host_u32(bk).T, want_bk)
        ix.sync()


@pytest.mark.parametrize("shards", [1, 3])
def test_optimal_insert_and_query(shards):
    s = _s()
    g = datagen.Generator()
    n = 20_000
    offs, cols = _with_edges(*g.rows(5, 0, n), 1 << 20)
    n = len(offs) - 1
    p = s.Params(K=4, L=16, log2_buckets=8, reservoir=32, cm_rows=4, cm_width=4096, shards=shards,
                 capacity=n + 3, seed=5, densify=1)
    ox = oracle.Index(K=4, L=16, log2_buckets=8, reservoir=32, cm_rows=4, cm_width=4096, shards=shards,
                      seed=5, capacity=n + 3, densify=1)
    ox.insert(offs, cols)
    want_slots, want_fill = ox.export()
    qo, qc, _ = g.queries(5, 6, 300, n)
    qo, qc = _with_edges(qo, qc, 1 << 20, seed=2)
    eids, esc = ox.query(qo, qc, 10)
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        slots, fill = ix.export()
        assert np.array_equal(fill, want_fill) and np.array_equal(slots, want_slots)
        for mode in ("fused", "plain"):
            ids, sc = ix.query(_dev(qo), _dev(qc), 10, mode=mode)
            assert np.array_equal(ids.cpu().numpy(), eids), mode
            assert np.array_equal(_host_u32(sc), esc), mode
        ix.sync()


def test_optimal_sketch_buckets():
    s = _s()
    g = datagen.Generator()
    n = 8000
    offs, cols = _with_edges(*g.rows(7, 0, n), 1 << 20)
    n = len(offs) - 1
    p = s.TkParams(K=4, L=16, log2_buckets=9, rows=4, cells=16, shards=2, seed=3, capacity=n, densify=1)
    ox = oracle.TkIndex(K=4, L=16, log2_buckets=9, rows=4, cells=16, shards=2, seed=3, capacity=n, densify=1)
    ox.insert(offs, cols)
    cells = ox.export()
    want = np.where(cells[..., 1] > 0, cells[..., 0] + 1, 0).astype(np.uint32)
    qo, qc, _ = g.queries(7, 8, 300, n)
    eids, esc = ox.query(qo, qc, 10)
    with s.TkIndex(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        assert np.array_equal(ix.export(), want)
        ids, sc = ix.query(_dev(qo), _dev(qc), 10)
        assert np.array_equal(ids.cpu().numpy(), eids)
        assert np.array_equal(_host_u32(sc), esc)
        ix.sync()

"""GPU parity of the TopKAPI sketch buckets (Sec. 3.1, Appendix 2) against the
oracle's sequential cell rule, bit-exact, through the C ABI."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from test_gpu_parity import _dev, _host_u32, _with_edges, _csr

pytestmark = pytest.mark.gpu


def _s():
    import paper_2008_03260_b300 as s
    return s


def _expected_words(ox: oracle.TkIndex) -> np.ndarray:
    cells = ox.export()
    hh, cnt = cells[..., 0], cells[..., 1]
    assert cnt.max() <= 1  # unique ids: a cell's count never passes 1
    return np.where(cnt > 0, hh + 1, 0).astype(np.uint32)


CONFIGS = [  # K, L, B, W, C, S   (W*C spans 1..32 cells per lane)
    (4, 16, 12, 4, 32, 1),
    (2, 8, 6, 1, 16, 1),
    (4, 16, 10, 2, 32, 3),
    (3, 7, 5, 8, 32, 2),
    (4, 16, 8, 8, 128, 1),
    (1, 1, 1, 3, 4, 1),
    (6, 64, 9, 4, 64, 1),
]


@pytest.mark.parametrize("K,L,B,W,C,S", CONFIGS)
def test_sketch_insert_and_query_match_oracle(K, L, B, W, C, S):
    s = _s()
    g = datagen.Generator()
    n = 6000
    offs, cols = g.rows(0, 0, n)
    offs, cols = _with_edges(offs, cols, 1 << 20)
    n = len(offs) - 1
    p = s.TkParams(K=K, L=L, log2_buckets=B, rows=W, cells=C, shards=S, seed=7, capacity=n + 5)
    ox = oracle.TkIndex(K=K, L=L, log2_buckets=B, rows=W, cells=C, shards=S, seed=7, capacity=n + 5)
    with s.TkIndex(p) as ix:
        # ragged batches: one row, a short run, the rest
        for a, b in [(0, 1), (1, 1000), (1000, n)]:
            o = offs[a:b + 1]
            first = ix.insert(_dev(o), _dev(cols))
            assert first == ox.insert(o - o[0], cols[int(o[0]):int(o[-1])])
        ix.sync()
        assert np.array_equal(ix.export(), _expected_words(ox))
        qo, qc, _ = g.queries(0, 1, 300, n, p_perturb=0.2)
        qo, qc = _with_edges(qo, qc, 1 << 20, seed=1)
        dq, dc = _dev(qo), _dev(qc)
        for k, thr in [(1, 0), (10, 0), (100, 0), (256, 0), (10, 2)]:
            ids, sc = ix.query(dq, dc, k, threshold=thr)
            ix.sync()
            eids, esc = ox.query(qo, qc, k, threshold=thr)
            assert np.array_equal(ids.cpu().numpy(), eids), (k, thr)
            assert np.array_equal(_host_u32(sc), esc), (k, thr)


def test_sketch_order_free_insert_and_reset():
    """Splitting the rows differently, or inserting again after a reset, gives the same cells."""
    s = _s()
    g = datagen.Generator()
    offs, cols = g.rows(3, 0, 5000)
    p = s.TkParams(K=4, L=16, log2_buckets=8, rows=4, cells=16, capacity=5000)
    with s.TkIndex(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        a = ix.export()
        ix.reset()
        assert ix.size == 0 and not ix.export().any()
        for r0 in range(0, 5000, 777):
            o = offs[r0:min(r0 + 777, 5000) + 1]
            ix.insert(_dev(o), _dev(cols))
        assert np.array_equal(ix.export(), a)


def test_sketch_errors():
    s = _s()
    with pytest.raises(s.SlashError):
        s.TkIndex(s.TkParams(rows=9, capacity=10))
    with pytest.raises(s.SlashError):
        s.TkIndex(s.TkParams(cells=24, capacity=10))
    with pytest.raises(s.SlashError):
        s.TkIndex(s.TkParams(rows=8, cells=256, capacity=10))  # 2048 cells per sketch
    p = s.TkParams(K=2, L=4, log2_buckets=4, rows=2, cells=8, capacity=3, dim=100)
    with s.TkIndex(p) as ix:
        offs, cols = _csr([np.array([1, 2], np.uint32), np.array([200], np.uint32)])
        ix.insert(_dev(offs), _dev(cols))
        with pytest.raises(s.SlashError) as e:
            ix.sync()
        assert e.value.code == s.SLASH_EDATA
        with pytest.raises(s.SlashError) as e:
            ix.insert(_dev(offs), _dev(cols))
        assert e.value.code == s.SLASH_EFULL
        assert ix.insert(_dev(np.zeros(1, np.uint64)), _dev(cols)) == 2  # empty batch: no-op
        ids, sc = ix.query(_dev(np.zeros(1, np.uint64)), _dev(cols), 5)
        assert ids.numel() == 0
        with pytest.raises(s.SlashError):
            ix.query(_dev(offs), _dev(cols), 0)


def test_heavy_sketch_paths():
    """12,000 copies of one row land in one sketch per table: with 2^24 sketches
    per table the rank field holds 255, so most copies take cursor slots, and
    the sketch's 12,000 staged ids go through the sliced merge.  Checked on the
    heavy sketches and on every sketch of 100 queries, against a partial oracle."""
    s = _s()
    g = datagen.Generator()
    base_o, base_c = g.rows(9, 0, 3000)
    rows = [base_c[int(base_o[i]):int(base_o[i + 1])] for i in range(3000)]
    heavy = rows[0]
    mixed = []
    for i in range(3000):
        mixed.append(rows[i])
        mixed.extend([heavy] * 4)
    offs, cols = _csr(mixed)
    n = len(offs) - 1
    K, L, B, W, C = 2, 2, 24, 2, 8
    qo, qc, _ = g.queries(9, 10, 100, 3000)
    _, qbk = oracle.hash_rows(K, L, B, 3, W, qo, qc, want_codes=False)
    _, hbk = oracle.hash_rows(K, L, B, 3, W, offs[:2], cols[:int(offs[1])], want_codes=False)
    rt = np.concatenate([np.tile(np.arange(L), 100), np.arange(L)]).astype(np.uint32)
    rb = np.concatenate([qbk.ravel(), hbk.ravel()]).astype(np.uint32)
    p = s.TkParams(K=K, L=L, log2_buckets=B, rows=W, cells=C, seed=3, capacity=n)
    with s.TkIndex(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        ids, sc = ix.query(_dev(qo), _dev(qc), 10)
        ix.sync()
        got = ix.buckets(np.zeros_like(rt), rt, rb)
    ox = oracle.TkIndex(K=K, L=L, log2_buckets=B, rows=W, cells=C, seed=3, capacity=n, partial=(rt, rb))
    ox.insert(offs, cols, threads=4)
    for i in range(len(rt)):
        cells = ox.bucket(int(rt[i]), int(rb[i]))
        assert np.array_equal(got[i], np.where(cells[..., 1] > 0, cells[..., 0] + 1, 0).astype(np.uint32)), i
    eids, esc = ox.query(qo, qc, 10)
    assert np.array_equal(ids.cpu().numpy(), eids)
    assert np.array_equal(_host_u32(sc), esc)

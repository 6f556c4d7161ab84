"""Pins of the oracle's TopKAPI buckets (Sec. 3.1 / Appendix 2) to properties
that do not depend on the oracle's own code."""
import numpy as np

import datagen
import oracle

EMPTY = 0xFFFFFFFF


def _run(stream):
    cell = (EMPTY, 0)
    for x in stream:
        cell = oracle.tk_update(cell, x)
    return cell


def test_cell_keeps_a_strict_majority():
    """A frequent-items cell: an element with a strict majority of a stream ends
    as the cell's heavy hitter, whatever the order (the Boyer-Moore guarantee)."""
    rng = np.random.default_rng(0)
    for _ in range(300):
        n = int(rng.integers(1, 40))
        maj = int(rng.integers(0, 1000))
        k = n // 2 + 1
        others = [int(v) for v in rng.integers(1000, 1100, n - k)]
        stream = [maj] * k + others
        rng.shuffle(stream)
        h, c = _run(stream)
        assert h == maj and 1 <= c <= k


def test_cell_single_element_and_distinct_streams():
    assert _run([7] * 13) == (7, 13)
    # distinct ids (every bucket stream, since ids are unique): each arrival meets
    # an empty cell or a different id with count 1, so the cell ends (last id, 1)
    rng = np.random.default_rng(1)
    for _ in range(100):
        stream = [int(v) for v in rng.choice(10**6, size=int(rng.integers(1, 60)), replace=False)]
        assert _run(stream) == (stream[-1], 1)


def test_merge_rules():
    assert oracle.tk_merge((EMPTY, 0), (5, 3)) == (5, 3)
    assert oracle.tk_merge((5, 3), (EMPTY, 0)) == (5, 3)
    assert oracle.tk_merge((5, 3), (5, 4)) == (5, 7)
    assert oracle.tk_merge((5, 3), (6, 1)) == (5, 2)
    assert oracle.tk_merge((5, 1), (6, 3)) == (6, 2)
    assert oracle.tk_merge((5, 2), (6, 2))[1] == 0          # equal counts cancel
    rng = np.random.default_rng(2)
    for _ in range(500):  # commutative up to the identity of an empty cell
        a = (int(rng.integers(0, 4)), int(rng.integers(0, 5)))
        b = (int(rng.integers(0, 4)), int(rng.integers(0, 5)))
        x, y = oracle.tk_merge(a, b), oracle.tk_merge(b, a)
        assert x[1] == y[1] and (x[1] == 0 or x[0] == y[0])


def test_merged_cells_keep_a_majority_holder():
    """Folding cells that each hold one id with count 1: an id holding the cell
    in more than half of the sketches is the merged heavy hitter."""
    rng = np.random.default_rng(3)
    for _ in range(300):
        n = int(rng.integers(1, 64))
        k = n // 2 + 1
        seq = [(9, 1)] * k + [(int(v), 1) for v in rng.integers(10, 20, n - k)]
        rng.shuffle(seq)
        acc = (EMPTY, 0)
        for cell in seq:
            acc = oracle.tk_merge(acc, cell)
        assert acc[0] == 9 and acc[1] >= 1


def test_sketch_index_shape_and_recall():
    """Buckets hold only ids hashed to them; planted neighbours are reported."""
    g = datagen.Generator()
    n = 4000
    offs, cols = g.rows(0, 0, n)
    ix = oracle.TkIndex(K=4, L=16, log2_buckets=12, rows=4, cells=32, capacity=n)
    ix.insert(offs, cols)
    cells = ix.export()
    _, bk = oracle.hash_rows(4, 16, 12, 0, 4, offs, cols, want_codes=False)
    occupied = cells[..., 1] > 0
    assert np.all(cells[..., 1][occupied] == 1)             # unique ids: counts stay 1
    hh = cells[..., 0][occupied]
    assert hh.max() < n
    # every kept id was hashed to that bucket
    s, t, b, r, c = np.nonzero(occupied)
    assert np.all(bk[cells[s, t, b, r, c, 0], t] == b)
    qo, qc, src = g.queries(0, 1, 300, n, p_perturb=0.2)
    ids, sc = ix.query(qo, qc, 10)
    assert np.mean([src[i] in ids[i] for i in range(300)]) > 0.85
    assert np.all(sc[:, 0] >= 1)


def test_threshold_filters_by_score():
    g = datagen.Generator()
    n = 3000
    offs, cols = g.rows(0, 0, n)
    ix = oracle.TkIndex(K=2, L=16, log2_buckets=8, rows=2, cells=16, capacity=n)
    ix.insert(offs, cols)
    qo, qc, _ = g.queries(0, 1, 100, n, p_perturb=0.1)
    ids0, sc0 = ix.query(qo, qc, 20)
    ids2, sc2 = ix.query(qo, qc, 20, threshold=2)
    for i in range(100):
        keep = [(a, b) for a, b in zip(ids0[i], sc0[i]) if a >= 0 and b > 2]
        got = [(a, b) for a, b in zip(ids2[i], sc2[i]) if a >= 0]
        assert got == keep
        assert np.all(ids2[i][len(got):] == -1) and np.all(sc2[i][len(got):] == 0)


def test_partial_parallel_insert_matches_dense():
    """The partial index with the parallel hash keeps exactly the dense
    index's cells for the listed sketches, and answers queries over them."""
    g = datagen.Generator()
    n = 5000
    offs, cols = g.rows(2, 0, n)
    qo, qc, _ = g.queries(2, 3, 40, n)
    dense = oracle.TkIndex(K=3, L=8, log2_buckets=7, rows=2, cells=8, shards=2, seed=4, capacity=n)
    dense.insert(offs, cols)
    _, qbk = oracle.hash_rows(3, 8, 7, 4, 2, qo, qc, want_codes=False)
    rt = np.concatenate([np.tile(np.arange(8), 40), np.arange(8)]).astype(np.uint32)
    rb = np.concatenate([qbk.ravel(), np.arange(8)]).astype(np.uint32)
    part = oracle.TkIndex(K=3, L=8, log2_buckets=7, rows=2, cells=8, shards=2, seed=4, capacity=n,
                          partial=(rt, rb))
    part.insert(offs[:2001], cols, threads=3)
    part.insert(offs[2000:] - offs[2000], cols[int(offs[2000]):], threads=2)
    full = dense.export()
    for t, b in zip(rt, rb):
        for s in range(2):
            assert np.array_equal(part.bucket(int(t), int(b), s), full[s, t, b])
    a, b_ = dense.query(qo, qc, 5)
    c, d = part.query(qo, qc, 5)
    assert np.array_equal(a, c) and np.array_equal(b_, d)


# ---------------------------------------------------------------------------- query report, worked by hand
# Appendix 2 "Querying": the merged sketch's heavy hitters are reported with
# their counts; an id may hold several cells (one per sketch row, or more), and
# this build scores it by the largest of its counts.  The expected values below
# are worked out by hand from the cells, not computed through the oracle.

def test_rank_scores_an_id_by_its_largest_cell():
    # id 7 holds two cells (counts 3 and 5), id 9 one cell (6), one cell is empty.
    #   largest count: 9 -> 6, 7 -> 5            => [(9, 6), (7, 5), pad]
    #   (a sum would rank 7 first with 8; the first cell would score 7 with 3)
    mh = [7, 9, 7, EMPTY]
    mc = [3, 6, 5, 0]
    ids, sc = oracle.tk_rank(mh, mc, 3)
    assert ids.tolist() == [9, 7, -1]
    assert sc.tolist() == [6, 5, 0]
    # the same cells in another order give the same report
    ids, sc = oracle.tk_rank([7, 7, EMPTY, 9], [5, 3, 0, 6], 3)
    assert ids.tolist() == [9, 7, -1] and sc.tolist() == [6, 5, 0]


def test_rank_ties_threshold_and_padding():
    # equal scores rank by smaller id; a score must exceed the threshold
    mh = [4, 3, 5, 4]
    mc = [2, 2, 1, 1]
    ids, sc = oracle.tk_rank(mh, mc, 4)
    assert ids.tolist() == [3, 4, 5, -1] and sc.tolist() == [2, 2, 1, 0]
    ids, sc = oracle.tk_rank(mh, mc, 4, threshold=1)
    assert ids.tolist() == [3, 4, -1, -1] and sc.tolist() == [2, 2, 0, 0]
    ids, sc = oracle.tk_rank(mh, mc, 2, threshold=2)
    assert ids.tolist() == [-1, -1] and sc.tolist() == [0, 0]
    # an id whose largest count passes the threshold is kept with that count,
    # even though another of its cells does not pass
    ids, sc = oracle.tk_rank([7, 7], [1, 4], 1, threshold=3)
    assert ids.tolist() == [7] and sc.tolist() == [4]
    # k smaller than the number of heavy hitters: only the first k
    ids, sc = oracle.tk_rank([1, 2, 3], [5, 9, 7], 2)
    assert ids.tolist() == [2, 3] and sc.tolist() == [9, 7]


def test_fold_follows_the_merge_rule_in_order():
    x, y, z = 11, 22, 33
    # one-cell sketches A = (x, 2), B = (y, 2), C = (z, 1)
    A, B, C = [[x, 2]], [[y, 2]], [[z, 1]]
    # A, B, C: (x,2) + (y,2) -> equal counts cancel -> empty; + (z,1) -> (z,1)
    mh, mc = oracle.tk_fold([A, B, C])
    assert (int(mh[0]), int(mc[0])) == (z, 1)
    # A, C, B: (x,2) + (z,1) -> x keeps 1; + (y,2) -> y wins with 2-1 = 1
    mh, mc = oracle.tk_fold([A, C, B])
    assert (int(mh[0]), int(mc[0])) == (y, 1)
    # same heavy hitter: counts add; an empty cell leaves the other unchanged
    mh, mc = oracle.tk_fold([[[x, 2], [EMPTY, 0]], [[x, 3], [y, 4]], [[EMPTY, 0], [y, 1]]])
    assert mh[0] == x and mc[0] == 5 and mh[1] == y and mc[1] == 5
    # nothing folded: every cell empty
    mh, mc = oracle.tk_fold(np.zeros((0, 3, 2), np.uint32))
    assert np.all(mc == 0)


def test_query_folds_shard_major_then_table_order():
    """The index query equals ranking the fold of its S*L sketches taken
    shard-major, then in table order; at least one query's answer changes when
    the sketches are folded table-major instead (so the order is checked)."""
    g = datagen.Generator()
    n = 6000
    offs, cols = g.rows(4, 0, n)
    S, L, B, W, C = 2, 8, 3, 2, 2
    ix = oracle.TkIndex(K=2, L=L, log2_buckets=B, rows=W, cells=C, shards=S, seed=6, capacity=n)
    ix.insert(offs, cols)
    qo, qc, _ = g.queries(4, 5, 60, n, p_perturb=0.2)
    ids, sc = ix.query(qo, qc, 6)
    _, qbk = oracle.hash_rows(2, L, B, 6, W, qo, qc, want_codes=False)
    differs = 0
    for q in range(60):
        sk = {(s, t): ix.bucket(t, int(qbk[q, t]), s).reshape(W * C, 2) for s in range(S) for t in range(L)}
        shard_major = [sk[(s, t)] for s in range(S) for t in range(L)]
        table_major = [sk[(s, t)] for t in range(L) for s in range(S)]
        a = oracle.tk_rank(*oracle.tk_fold(shard_major), 6)
        assert np.array_equal(a[0], ids[q]) and np.array_equal(a[1], sc[q])
        b = oracle.tk_rank(*oracle.tk_fold(table_major), 6)
        differs += not (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]))
    assert differs > 0

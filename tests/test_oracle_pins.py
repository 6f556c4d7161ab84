"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each oracle function is tied to a published test vector, a closed form from
the paper, an invariant of the data structure, or a brute-force definition on
tiny inputs -- chosen so that a plausible slip (a dropped term, a wrong side,
a transposed operand) fails at least one test here.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M32 = 0xFFFFFFFF
M31 = 0x7FFFFFFF


def _rows(path):
    with open(os.path.join(GOLDEN, path)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------------ primitives
def test_mix32_published_vectors():
    """MurmurHash3_x86_32 of the empty key is fmix32(seed): SMHasher's values."""
    for a, b in _rows("murmur3_fmix32.txt"):
        assert oracle.mix32(int(a, 16)) == int(b, 16)


def _unmix(y, bits):
    """Inverse of the finaliser, derived step by step (xor-shift and odd multiply)."""
    m = (1 << bits) - 1
    y &= m
    y ^= y >> 16
    y = (y * pow(0xC2B2AE35 & m, -1, 1 << bits)) & m
    y ^= (y >> 13) ^ (y >> 26)
    y = (y * pow(0x85EBCA6B & m, -1, 1 << bits)) & m
    y ^= y >> 16
    return y


def test_mix32_and_mix31_are_bijections():
    """An independently derived inverse undoes them; mix31 stays inside 31 bits."""
    rng = np.random.default_rng(1)
    xs = [0, 1, 2, M31, M32, 0x80000000] + [int(v) for v in rng.integers(0, 1 << 32, 3000)]
    for x in xs:
        assert _unmix(oracle.mix32(x), 32) == x
        y = oracle.mix31(x)
        assert y <= M31
        assert _unmix(y, 31) == x & M31


def test_splitmix64_published_vectors():
    for row in _rows("splitmix64.txt"):
        seed, outs = int(row[0]), [int(v) for v in row[1:]]
        assert oracle.splitmix64_stream(seed, len(outs)) == outs


def test_seed_derivation_order():
    """Sub-seeds are the upper halves of SplitMix64 outputs in the stated order."""
    outs = [int(v) for v in _rows("splitmix64.txt")[0][1:]]
    s = oracle.derive_seeds(0, 3, 2)
    assert s["a"] == outs[0] >> 32 and s["dirseed"] == outs[1] >> 32
    assert int(s["st"][0]) == outs[2] >> 32
    assert len(s["st"]) == 3 and len(s["sp"]) == 3 and len(s["sc"]) == 2


# ------------------------------------------------------------------ MinHash / DOPH
def test_doph_single_bin_is_plain_minhash():
    """nb = 1: no binning, no densification -- DOPH is MinHash, min over pi(i) (Sec. 2.2)."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        cols = rng.choice(1 << 20, size=int(rng.integers(1, 60)), replace=False)
        a = int(rng.integers(0, 1 << 32))
        codes, mask = oracle.doph(cols, 1, a, 123)
        assert codes[0] == min(oracle.mix32(int(c) ^ a) for c in cols)
        assert codes[0] == oracle.minhash(cols, a)
        assert mask[0]


def _doph_brute(cols, nb, a, dirseed):
    """Sec. 2.2 written out with explicit loops: range bins, per-bin minimum, then
    every empty bin walks to the closest non-empty bin on its (seeded) side."""
    h = {int(c): oracle.mix32(int(c) ^ a) for c in cols}
    m = [None] * nb
    for c, v in h.items():
        j = (v * nb) >> 32
        m[j] = v if m[j] is None else min(m[j], v)
    if all(v is None for v in m):
        return [M32] * nb, [False] * nb
    out = []
    for j in range(nb):
        if m[j] is not None:
            out.append(m[j])
            continue
        step = 1 if oracle.mix32(j ^ dirseed) & 1 else -1
        k = j
        while True:
            k = (k + step) % nb
            if m[k] is not None:
                break
        out.append(m[k])
    return out, [v is not None for v in m]


@pytest.mark.parametrize("nb", [1, 2, 7, 32, 64, 100, 384])
def test_doph_brute_force(nb):
    rng = np.random.default_rng(nb)
    for trial in range(40):
        n = int(rng.integers(0, 50)) if trial else 0
        cols = rng.choice(1 << 20, size=n, replace=False)
        if trial % 7 == 3 and n:  # duplicates in a row do not change a set function
            cols = np.concatenate([cols, cols[: n // 2]])
        a, ds = (int(v) for v in rng.integers(0, 1 << 32, 2))
        codes, mask = oracle.doph(cols, nb, a, ds)
        want, wmask = _doph_brute(cols, nb, a, ds)
        assert list(codes) == want
        assert list(mask) == wmask


def _pair(rng, n, s):
    """Two sets of size n sharing s features: Jaccard = s / (2n - s)."""
    f = rng.choice(1 << 20, size=2 * n - s, replace=False)
    return f[:n], np.concatenate([f[:s], f[n:]])


@pytest.mark.parametrize("n,s", [(22, 4), (30, 20), (36, 32), (39, 38)])
def test_doph_collision_probability_is_jaccard(n, s):
    """Sec. 2.2: P[h(x) = h(y)] is the Jaccard index (the printed fraction's sign is
    garbled; x.y / (|x| + |y| - x.y) is read).  With densification every one of
    the nb bins keeps that collision probability; nb = 64 > n forces ~half of
    the bins of each row to be densified."""
    J = s / (2 * n - s)
    nb, T = 64, 1500
    rng = np.random.default_rng(1000 + n)
    hits = np.zeros(nb)
    both_empty_hits = 0
    both_empty = 0
    for t in range(T):
        x, y = _pair(rng, n, s)
        a, ds = (int(v) for v in rng.integers(0, 1 << 32, 2))
        cx, mx = oracle.doph(x, nb, a, ds)
        cy, my = oracle.doph(y, nb, a, ds)
        eq = cx == cy
        hits += eq
        e = ~mx & ~my
        both_empty += e.sum()
        both_empty_hits += (eq & e).sum()
    sd = np.sqrt(J * (1 - J) / T)
    assert np.all(np.abs(hits / T - J) < 5 * sd + 1e-9), (hits / T, J)
    assert abs(hits.mean() / T - J) < 3 * sd
    # densified bins on their own also collide with probability J
    assert both_empty > 1000
    assert abs(both_empty_hits / both_empty - J) < 5 * np.sqrt(J * (1 - J) / both_empty)


def test_table_address_collision_closed_form():
    """Sec. 2.3 / Appendix 1: a table address collides when all K codes do, plus
    a 2^-B chance collision otherwise; and P[all K equal] >= J^K (the bound the
    proof uses, its printed inequalities read with the sides swapped)."""
    n, s = 36, 32  # J = 0.8
    J, K, L, B, T = s / (2 * n - s), 3, 8, 3, 1200
    rng = np.random.default_rng(7)
    allk = 0
    same = 0
    for t in range(T):
        x, y = _pair(rng, n, s)
        seed = int(rng.integers(0, 1 << 63))
        cx, bx = oracle.hash_rows(K, L, B, seed, 1, np.array([0, n], np.uint64), x)
        cy, by = oracle.hash_rows(K, L, B, seed, 1, np.array([0, n], np.uint64), y)
        eqk = (cx[0].reshape(L, K) == cy[0].reshape(L, K)).all(axis=1)
        allk += eqk.sum()
        same += (bx[0] == by[0]).sum()
    N = T * L
    pk, pb = allk / N, same / N
    pred = pk + (1 - pk) * 2.0 ** -B
    assert abs(pb - pred) < 4 * np.sqrt(pred * (1 - pred) / N)
    assert pk > J ** K - 4 * np.sqrt(J ** K * (1 - J ** K) / N)
    # all-equal codes always give the same address (same K codes, same table seed)
    assert pb >= pk


def test_table_address_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(200):
        K, B = int(rng.integers(1, 9)), int(rng.integers(1, 31))
        codes = [int(v) for v in rng.integers(0, 1 << 32, K * 3)]
        t = int(rng.integers(0, 3))
        st = int(rng.integers(0, 1 << 32))
        acc = st
        for j in range(K):
            acc = ((acc ^ codes[t * K + j]) * 0x9E3779B1) & M32
        assert oracle.table_address(codes, t, K, B, st) == oracle.mix32(acc) >> (32 - B)
        # changing one of the table's codes moves the address (almost surely) ...
        c2 = list(codes)
        c2[t * K] ^= 1
        assert oracle.table_address(c2, t, K, 30, st) != oracle.table_address(codes, t, K, 30, st) or B < 30
        # ... and another table's codes never matter
        c3 = list(codes)
        c3[((t + 1) % 3) * K] ^= 0xDEADBEEF
        assert oracle.table_address(c3, t, K, B, st) == oracle.table_address(codes, t, K, B, st)


# ------------------------------------------------------------------ reservoir buckets
def _small_index(n_rows, **kw):
    import datagen
    g = datagen.Generator()
    offs, cols = g.rows(kw.pop("data_seed", 0), 0, n_rows)
    p = dict(K=2, L=4, log2_buckets=3, reservoir=5, cm_rows=3, cm_width=64, capacity=n_rows)
    p.update(kw)
    return offs, cols, p


def test_reservoir_brute_force():
    """Every bucket holds the R ids of smallest priority among all ids hashed to
    it, ascending -- checked against an explicit sort of each bucket's ids."""
    offs, cols, p = _small_index(400)
    ix = oracle.Index(**p)
    ix.insert(offs, cols)
    slots, fill = ix.export()
    _, bk = oracle.hash_rows(p["K"], p["L"], p["log2_buckets"], 0, p["cm_rows"], offs, cols, False)
    sp = oracle.derive_seeds(0, p["L"], p["cm_rows"])["sp"]
    R = p["reservoir"]
    overflow = 0
    for t in range(p["L"]):
        for b in range(1 << p["log2_buckets"]):
            ids = [i for i in range(400) if bk[i, t] == b]
            ids.sort(key=lambda i: oracle.priority(i, int(sp[t])))
            overflow += len(ids) > R
            keep = ids[:R]
            assert fill[0, t, b] == len(keep)
            assert list(slots[0, t, b, :len(keep)]) == keep
            assert np.all(slots[0, t, b, len(keep):] == oracle.EMPTY)
    assert overflow > 0  # the check covered sub-sampled (full) buckets


def test_reservoir_order_and_batch_invariance():
    """The bucket contents do not depend on insertion order or batching: three
    uneven batches, and a threaded insert that merges private reservoirs, give
    the same index as one sequential pass."""
    offs, cols, p = _small_index(3000, log2_buckets=6, reservoir=7)
    one = oracle.Index(**p)
    one.insert(offs, cols)
    s1, f1 = one.export()
    three = oracle.Index(**p)
    for a, b in [(0, 17), (17, 1900), (1900, 3000)]:
        o = offs[a:b + 1]
        three.insert(o, cols[int(o[0]):int(o[-1])])
    s3, f3 = three.export()
    assert np.array_equal(s1, s3) and np.array_equal(f1, f3)
    tt, bb = np.meshgrid(np.arange(p["L"]), np.arange(1 << p["log2_buckets"]), indexing="ij")
    par = oracle.Index(**p, partial=(tt.ravel(), bb.ravel()))
    par.insert(offs, cols, threads=5)
    for t in range(p["L"]):
        for b in range(1 << p["log2_buckets"]):
            s, f = par.bucket(t, b)
            assert f == f1[0, t, b] and np.array_equal(s, s1[0, t, b])


# ------------------------------------------------------------------ sketch and ranking
def _query_details(shards=1, n_rows=1500, w=64, R=6, **kw):
    import datagen
    offs, cols, p = _small_index(n_rows, log2_buckets=4, reservoir=R, cm_width=w, shards=shards, **kw)
    ix = oracle.Index(**p)
    ix.insert(offs, cols)
    g = datagen.Generator()
    qo, qc, _ = g.queries(0, 5, 40, n_rows, p_perturb=0.3)
    return ix, p, [ix.query_detail(qc[int(qo[i]):int(qo[i + 1])], 10) for i in range(40)]


def test_countmin_invariants():
    """Count-min (named in Sec. 3.1): every row of the sketch sums to |M|; the
    estimate never falls below the exact count; it equals the exact count when
    one of the id's cells is shared with no other candidate."""
    ix, p, dets = _query_details()
    sc = oracle.derive_seeds(0, p["L"], p["cm_rows"])["sc"]
    eq_cases = 0
    for d in dets:
        M, U = d["M"], d["U"]
        assert np.all(d["cm"].sum(axis=1) == len(M))
        assert np.array_equal(U, np.unique(M))
        cnt = np.array([(M == u).sum() for u in U])
        assert np.array_equal(d["cnt"], cnt)
        assert np.all(d["est"] >= cnt)
        assert np.all(cnt <= p["L"] * p["shards"])
        cells = np.array([[oracle.cm_cell(int(u), int(sc[r]), p["cm_width"]) for r in range(p["cm_rows"])]
                          for u in U]).reshape(len(U), p["cm_rows"])
        for i in range(len(U)):
            alone = [r for r in range(p["cm_rows"]) if (cells[:, r] == cells[i, r]).sum() == 1]
            if alone:
                eq_cases += 1
                assert d["est"][i] == cnt[i]
    assert eq_cases > 100


def test_topk_ranking_brute_force():
    """Sec. 2.3 frequency ranking: estimate descending, ties by smaller id, -1/0 padding."""
    for w, R in [(64, 6), (32, 2)]:
        _, _, dets = _query_details(w=w, R=R)
        padded = 0
        for d in dets:
            order = sorted(zip(d["U"].tolist(), d["est"].tolist()), key=lambda x: (-x[1], x[0]))[:10]
            ids = [i for i, _ in order] + [-1] * (10 - len(order))
            sc = [e for _, e in order] + [0] * (10 - len(order))
            assert list(d["ids"]) == ids and list(d["scores"]) == sc
            padded += len(order) < 10
        if R == 2:
            assert padded > 0


def test_shards_equal_one_index_without_subsampling():
    """Sec. 3: with shared seeds the partitions form one logical index.  When no
    bucket overflows, an S-shard index answers exactly like a 1-shard index over
    the same rows (sketches add; candidate sets unite)."""
    import datagen
    g = datagen.Generator()
    n = 2500
    offs, cols = g.rows(0, 0, n)
    qo, qc, _ = g.queries(0, 9, 200, n, p_perturb=0.2)
    base = dict(K=4, L=16, log2_buckets=16, reservoir=256, cm_rows=4, cm_width=4096, capacity=n)
    outs = []
    for S in (1, 4, 7):
        ix = oracle.Index(**base, shards=S)
        ix.insert(offs, cols)
        _, fill = ix.export()
        assert fill.max() < 256
        outs.append(ix.query(qo, qc, 10))
    for ids, sc in outs[1:]:
        assert np.array_equal(ids, outs[0][0]) and np.array_equal(sc, outs[0][1])


def test_shard_sketch_is_sum_of_partition_sketches():
    """Algorithm 2's cross-machine merge: the query sketch equals the cell-wise
    sum of the sketches each shard builds from its own buckets."""
    ix, p, dets = _query_details(shards=3, n_rows=1200)
    sc = oracle.derive_seeds(0, p["L"], p["cm_rows"])["sc"]
    for d in dets[:10]:
        cm = np.zeros((p["cm_rows"], p["cm_width"]), np.int64)
        for u in d["M"]:
            for r in range(p["cm_rows"]):
                cm[r, oracle.cm_cell(int(u), int(sc[r]), p["cm_width"])] += 1
        assert np.array_equal(cm, d["cm"])


def test_planted_recall_matches_binomial_model():
    """Appendix 1: a row found with per-table probability P_x appears in
    f_x ~ Binomial(L, P_x) of the query's buckets, P_x >= J^K.  Planted queries
    must be recalled at least as often as 1 - (1 - J^K)^L predicts, and their
    top-1 must mostly be the exact Jaccard nearest neighbour (brute force)."""
    import datagen
    g = datagen.Generator()
    n, nq, K, L = 3000, 400, 4, 16
    offs, cols = g.rows(0, 0, n)
    qo, qc, src = g.queries(0, 1, nq, n, p_perturb=0.2)
    ix = oracle.Index(K=K, L=L, log2_buckets=16, reservoir=32, cm_rows=4, cm_width=4096, capacity=n)
    ix.insert(offs, cols)
    ids, _ = ix.query(qo, qc, 10)
    rows = [set(cols[int(offs[i]):int(offs[i + 1])].tolist()) for i in range(n)]
    qs = [set(qc[int(qo[i]):int(qo[i + 1])].tolist()) for i in range(nq)]
    J = np.array([len(q & rows[s]) / len(q | rows[s]) for q, s in zip(qs, src)])
    p = 1 - (1 - J ** K) ** L
    recall = np.mean([src[i] in ids[i] for i in range(nq)])
    assert recall >= p.mean() - 3 * np.sqrt((p * (1 - p)).sum()) / nq
    nn_top1 = 0
    for i in range(100):
        js = [len(qs[i] & r) / len(qs[i] | r) for r in rows]
        nn_top1 += int(np.argmax(js)) == ids[i, 0]
    assert nn_top1 >= 85


# ---------------------------------------------------------------------------- exact neighbours (ground truth)
def _jaccard_brute(rows, q):
    qs = set(int(v) for v in q)
    out = []
    for i, r in enumerate(rows):
        rs = set(int(v) for v in r)
        u = len(qs | rs)
        out.append((Fraction(len(qs & rs), u) if u else Fraction(0), i))
    out.sort(key=lambda t: (-t[0], t[1]))
    return out


def test_jaccard_topk_against_python_sets():
    """The brute-force neighbours equal a Python-set computation of the
    similarity (exact fractions), ties by id, on random small sets."""
    rng = np.random.default_rng(11)
    dim = 256
    rows = [np.sort(rng.choice(dim, int(rng.integers(0, 12)), replace=False)).astype(np.uint32) for _ in range(300)]
    qs = [np.sort(rng.choice(dim, int(rng.integers(0, 12)), replace=False)).astype(np.uint32) for _ in range(40)]
    qs[0] = rows[17].copy()                      # a copy of a row: similarity 1
    qs[1] = np.zeros(0, np.uint32)               # empty query: similarity 0 to all
    offs = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.uint64)
    qo = np.concatenate([[0], np.cumsum([len(q) for q in qs])]).astype(np.uint64)
    ids, inter, uni = oracle.jaccard_topk(offs, np.concatenate(rows), qo, np.concatenate(qs), 7, dim=dim, threads=3)
    for qi, q in enumerate(qs):
        want = _jaccard_brute(rows, q)[:7]
        assert [i for _, i in want] == ids[qi].tolist(), qi
        for j, (f, _) in enumerate(want):
            got = Fraction(int(inter[qi, j]), int(uni[qi, j])) if uni[qi, j] else Fraction(0)
            assert got == f
    assert ids[0, 0] == 17 and inter[0, 0] == uni[0, 0] == len(rows[17])
    assert ids[1].tolist() == list(range(7))     # all similarities 0: smallest ids

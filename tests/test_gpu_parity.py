"""GPU parity: the CUDA path against the CPU oracle, bit-exact (integer work).

Everything goes through the C ABI (libslash.so) via the thin binding.  Inputs
come from the seeded generator; expected values only from ``oracle``.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu

EMPTY = 0xFFFFFFFF


def _dev(a: np.ndarray) -> torch.Tensor:
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host_u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def _slash():
    import paper_2008_03260_b300 as s
    return s


def _edge_rows(dim: int, rng) -> list[np.ndarray]:
    return [
        np.zeros(0, np.uint32),                                  # empty row
        np.array([dim - 1], np.uint32),                          # one feature, the last id
        np.full(10, 12345, np.uint32),                           # one feature, duplicated
        np.array([0, dim - 1, 0, 17, 17], np.uint32),            # unsorted + duplicates
        rng.choice(dim, 2000, replace=False).astype(np.uint32),  # widest query rows
        np.sort(rng.choice(dim, 200, replace=False)).astype(np.uint32)[::-1].copy(),
    ]


def _csr(rows: list[np.ndarray]):
    offs = np.zeros(len(rows) + 1, np.uint64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    cols = np.concatenate(rows).astype(np.uint32) if rows else np.zeros(0, np.uint32)
    return offs, cols


def _with_edges(offs, cols, dim, seed=0):
    rng = np.random.default_rng(seed)
    rows = [cols[int(offs[i]):int(offs[i + 1])] for i in range(len(offs) - 1)]
    e = _edge_rows(dim, rng)
    return _csr(e[:3] + rows[:len(rows) // 2] + e[3:] + rows[len(rows) // 2:])


@pytest.mark.parametrize("K,L,B", [(4, 16, 16), (6, 64, 18), (8, 32, 20), (3, 7, 5), (1, 1, 1), (16, 64, 20),
                                   (1, 1, 28)])
def test_hash_codes_and_addresses(K, L, B):
    s = _slash()
    g = datagen.Generator()
    offs, cols = _with_edges(*g.rows(3, 0, 3000), 1 << 20)
    p = s.Params(K=K, L=L, log2_buckets=B, reservoir=4, cm_rows=2, cm_width=64, capacity=10_000, seed=11)
    with s.Index(p) as ix:
        codes, bk = ix.debug_hash(_dev(offs), _dev(cols))
        torch.cuda.synchronize()
        want_codes, want_bk = oracle.hash_rows(K, L, B, 11, 2, offs, cols)
        assert np.array_equal(_host_u32(codes), want_codes)
        assert np.array_equal(_host_u32(bk).T, want_bk)
        assert ix.sync() is None


def _oracle_index(p, offs, cols, batches=None):
    ix = oracle.Index(K=p.K, L=p.L, log2_buckets=p.log2_buckets, reservoir=p.reservoir, cm_rows=p.cm_rows,
                      cm_width=p.cm_width, shards=p.shards, seed=p.seed, capacity=p.capacity)
    ix.insert(offs, cols)
    return ix


def _gpu_insert(ix, offs, cols, batches):
    """insert rows in the given batch boundaries; returns first ids"""
    firsts = []
    d_cols = _dev(cols)
    for a, b in zip(batches[:-1], batches[1:]):
        firsts.append(ix.insert(_dev(offs[a:b + 1]), d_cols))
    return firsts


@pytest.mark.parametrize("B,R,n", [(6, 32, 20_000), (4, 1, 5_000), (8, 512, 60_000), (16, 32, 30_000),
                                   (2, 200, 9_000)])
def test_insert_full_index_bit_exact(B, R, n):
    """Small tables force heavy sub-sampling (warp-sort and radix-select merges)."""
    s = _slash()
    g = datagen.Generator()
    offs, cols = _with_edges(*g.rows(5, 0, n), 1 << 20, seed=B)
    p = s.Params(K=4, L=16, log2_buckets=B, reservoir=R, cm_rows=4, cm_width=4096, capacity=n + 10, seed=5)
    want_slots, want_fill = _oracle_index(p, offs, cols).export()
    with s.Index(p) as ix:
        nr = len(offs) - 1
        assert _gpu_insert(ix, offs, cols, [0, nr]) == [0]
        ix.sync()
        slots, fill = ix.export()
    assert np.array_equal(fill, want_fill)
    assert np.array_equal(slots, want_slots)


def test_insert_batching_and_reinsertion_bit_exact():
    """Uneven batches (incl. one row and an empty batch) give the oracle's one-pass index."""
    s = _slash()
    g = datagen.Generator()
    n = 40_000
    offs, cols = g.rows(9, 0, n)
    p = s.Params(K=4, L=16, log2_buckets=7, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=9)
    want_slots, want_fill = _oracle_index(p, offs, cols).export()
    with s.Index(p) as ix:
        firsts = _gpu_insert(ix, offs, cols, [0, 1, 1, 777, 20_000, 39_999, n])
        assert firsts == [0, 1, 1, 777, 20_000, 39_999]
        ix.sync()
        slots, fill = ix.export()
        assert ix.size == n
    assert np.array_equal(fill, want_fill) and np.array_equal(slots, want_slots)


def _queries(g, n_rows, nq, seed=1, **kw):
    qo, qc, _ = g.queries(0, seed, nq, n_rows, **kw)
    return _with_edges(qo, qc, 1 << 20, seed=seed)


@pytest.mark.parametrize("topk", [10, 1, 100, 256])
def test_query_tiny_workload_bit_exact(topk):
    """The `tiny` workload at full size: 100k rows, 1000 planted queries + edge rows."""
    from datagen.workloads import TINY as w
    s = _slash()
    g = datagen.Generator()
    offs, cols = g.rows(w.seed, 0, w.n_rows)
    qo, qc = _queries(g, w.n_rows, w.n_queries, p_perturb=w.p_perturb)
    p = s.Params(**w.params())
    oix = _oracle_index(p, offs, cols)
    want_ids, want_sc = oix.query(qo, qc, topk)
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        ids, sc = ix.query(_dev(qo), _dev(qc), topk)
        ix.sync()
        assert np.array_equal(ids.cpu().numpy(), want_ids)
        assert np.array_equal(_host_u32(sc), want_sc)
        if topk <= 10:
            for mode in ("warp_fused", "warp_plain"):
                ids, sc = ix.query(_dev(qo), _dev(qc), topk, mode=mode)
                ix.sync()
                assert np.array_equal(ids.cpu().numpy(), want_ids), mode
                assert np.array_equal(_host_u32(sc), want_sc), mode
        slots, fill = ix.export()
    ws, wf = oix.export()
    assert np.array_equal(fill, wf) and np.array_equal(slots, ws)


@pytest.mark.parametrize("shards,R,B", [(8, 32, 16), (3, 8, 6), (8, 64, 10)])
def test_query_sharded_bit_exact(shards, R, B):
    """Sec. 3 partitions as on-device shards; query sketches summed across shards."""
    s = _slash()
    g = datagen.Generator()
    n = 30_000
    offs, cols = g.rows(2, 0, n)
    qo, qc = _queries(g, n, 500, seed=3, planted_frac=0.3, p_perturb=0.2)
    p = s.Params(K=4, L=16, log2_buckets=B, reservoir=R, cm_rows=4, cm_width=8192, shards=shards,
                 capacity=n, seed=2)
    oix = _oracle_index(p, offs, cols)
    want_ids, want_sc = oix.query(qo, qc, 10)
    with s.Index(p) as ix:
        _gpu_insert(ix, offs, cols, [0, 5000, 5001, n])
        ids, sc = ix.query(_dev(qo), _dev(qc), 10)
        ix.sync()
        # 256-thread teams: at (3, 8, 6) a CTA holds three of them (its TMEM allocation
        # is rounded up to a power of two); the warp engine hands its large queries to them
        for mode, thr in (("warp_fused", 256), ("warp_plain", 256), ("fused", 256), ("plain", 256)):
            wi, ws_ = ix.query(_dev(qo), _dev(qc), 10, mode=mode, threads=thr)
            ix.sync()
            assert np.array_equal(wi.cpu().numpy(), ids.cpu().numpy()), mode
            assert np.array_equal(_host_u32(ws_), _host_u32(sc)), mode
        slots, fill = ix.export()
    ws, wf = oix.export()
    assert np.array_equal(fill, wf) and np.array_equal(slots, ws)
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(_host_u32(sc), want_sc)


def test_query_heavy_collisions_and_capped_estimates():
    """A 32-wide sketch with 8 shards x 64 tables: estimates far above the exact
    counts and above the 255 histogram cap exercise the tie-break paths."""
    s = _slash()
    g = datagen.Generator()
    n = 20_000
    offs, cols = g.rows(4, 0, n)
    qo, qc = _queries(g, n, 300, seed=8)
    p = s.Params(K=2, L=64, log2_buckets=3, reservoir=16, cm_rows=1, cm_width=32, shards=8,
                 capacity=n, seed=4)
    oix = _oracle_index(p, offs, cols)
    want_ids, want_sc = oix.query(qo, qc, 50)
    assert want_sc.max() >= 255
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        ids, sc = ix.query(_dev(qo), _dev(qc), 50)
        ix.sync()
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(_host_u32(sc), want_sc)


@pytest.mark.parametrize("shards,L,R,d", [(1, 128, 128, 1), (4, 64, 32, 1), (2, 64, 64, 2)])
def test_query_capped_bin_decides_top10(shards, L, R, d):
    """k = 10 with a 32-wide sketch and up to 16k candidate occurrences: most
    estimates reach the 255 cap, so the cap bin alone decides the top-k.  Where
    its pool would outgrow the bound of the staged query, that query is
    answered again by the general one; both paths against the oracle."""
    s = _slash()
    g = datagen.Generator()
    n = 20_000
    offs, cols = g.rows(21, 0, n)
    qo, qc = _queries(g, n, 200, seed=22)
    p = s.Params(K=2, L=L, log2_buckets=3, reservoir=R, cm_rows=d, cm_width=32, shards=shards, capacity=n, seed=21)
    want_ids, want_sc = _oracle_index(p, offs, cols).query(qo, qc, 10)
    assert want_sc.max() >= 255
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        for mode in ("fused", "plain", "warp_fused", "warp_plain"):
            ids, sc = ix.query(_dev(qo), _dev(qc), 10, mode=mode)
            ix.sync()
            assert np.array_equal(ids.cpu().numpy(), want_ids), mode
            assert np.array_equal(_host_u32(sc), want_sc), mode


def test_query_few_distinct_ids_many_occurrences_pads():
    """One row inserted many times: its query meets more than 64 occurrences of
    fewer than k distinct ids, so the top-10 is padded with (-1, 0)."""
    s = _slash()
    g = datagen.Generator()
    offs, cols = g.rows(23, 0, 300)
    row = cols[int(offs[7]):int(offs[8])]
    rows = [cols[int(offs[i]):int(offs[i + 1])] for i in range(300)]
    rows = rows[:50] + [row] * 6 + rows[50:]
    o2, c2 = _csr(rows)
    qo, qc = _csr([row, row[: len(row) // 2], np.zeros(0, np.uint32)])
    p = s.Params(K=4, L=16, log2_buckets=16, reservoir=32, cm_rows=4, cm_width=4096, capacity=1000, seed=23)
    want_ids, want_sc = _oracle_index(p, o2, c2).query(qo, qc, 10)
    assert (want_ids[0] == -1).any() and want_ids[0][0] >= 0
    with s.Index(p) as ix:
        ix.insert(_dev(o2), _dev(c2))
        for mode in ("fused", "plain", "warp_fused", "warp_plain"):
            ids, sc = ix.query(_dev(qo), _dev(qc), 10, mode=mode)
            ix.sync()
            assert np.array_equal(ids.cpu().numpy(), want_ids), mode
            assert np.array_equal(_host_u32(sc), want_sc), mode


def test_invalid_columns_are_skipped_and_reported():
    s = _slash()
    g = datagen.Generator()
    offs, cols = g.rows(6, 0, 2000)
    bad = cols.copy()
    bad[5] = 1 << 20
    bad[900] = 0xFFFFFFFF
    keep = np.ones(len(cols), bool)
    keep[[5, 900]] = False
    rows = [cols[int(offs[i]):int(offs[i + 1])][keep[int(offs[i]):int(offs[i + 1])]] for i in range(2000)]
    goffs, gcols = _csr(rows)
    p = s.Params(K=4, L=16, log2_buckets=8, reservoir=8, cm_rows=4, cm_width=4096, capacity=4000, seed=6)
    want_slots, want_fill = _oracle_index(p, goffs, gcols).export()
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(bad))
        assert s.slash_sync(ix.h) == s.SLASH_EDATA
        assert s.slash_sync(ix.h) == s.SLASH_OK  # cleared
        slots, fill = ix.export()
    assert np.array_equal(fill, want_fill) and np.array_equal(slots, want_slots)


def test_argument_errors():
    s = _slash()
    p = s.Params(K=4, L=16, log2_buckets=8, reservoir=8, cm_rows=4, cm_width=4096, capacity=10, seed=6)
    g = datagen.Generator()
    offs, cols = g.rows(6, 0, 11)
    with s.Index(p) as ix:
        with pytest.raises(s.SlashError) as e:
            ix.insert(_dev(offs), _dev(cols))
        assert e.value.code == s.SLASH_EFULL
        assert ix.size == 0
        ix.insert(_dev(offs[:11]), _dev(cols))
        assert ix.size == 10
        for k in (0, 257):
            with pytest.raises(s.SlashError) as e:
                ix.query(_dev(offs), _dev(cols), k)
            assert e.value.code == s.SLASH_EINVAL
        ids, sc = ix.query(_dev(offs[:1]), _dev(cols), 5)  # zero queries
        assert ids.numel() == 0
        ix.reset()
        assert ix.size == 0
        slots, fill = ix.export()
        assert fill.max() == 0 and np.all(slots == EMPTY)


@pytest.mark.parametrize("shards,R,B,w,topk", [(1, 32, 16, 4096, 20), (8, 16, 8, 8192, 20), (2, 128, 12, 1024, 20),
                                                (1, 32, 16, 4096, 10), (8, 16, 8, 8192, 10), (2, 128, 12, 1024, 7),
                                                (4, 30, 9, 2048, 10)])
def test_every_query_schedule_is_bit_exact(shards, R, B, w, topk):
    """Fused persistent and plain per-stage kernels, every CTA size and CTAs/SM
    cap: the same ids and scores as the oracle (integer work, tolerance zero)."""
    s = _slash()
    g = datagen.Generator()
    n = 25_000
    offs, cols = g.rows(12, 0, n)
    qo, qc = _queries(g, n, 700, seed=13, planted_frac=0.3, p_perturb=0.2)
    p = s.Params(K=4, L=16, log2_buckets=B, reservoir=R, cm_rows=4, cm_width=w, shards=shards,
                 capacity=n, seed=12)
    want_ids, want_sc = _oracle_index(p, offs, cols).query(qo, qc, topk)
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        dq, dc = _dev(qo), _dev(qc)
        for mode in ("fused", "plain", "warp_fused", "warp_plain"):
            for threads in (256, 512, 1024):
                for cps in (0, 1):
                    if mode.startswith("warp") and (topk > 10 or threads != 256):
                        if topk > 10:  # the warp schedules serve k <= 10 only
                            with pytest.raises(s.SlashError) as e:
                                ix.query(dq, dc, topk, mode=mode, threads=threads, ctas_per_sm=cps)
                            assert e.value.code == s.SLASH_EINVAL
                        continue
                    ids, sc = ix.query(dq, dc, topk, mode=mode, threads=threads, ctas_per_sm=cps)
                    ix.sync()
                    assert np.array_equal(ids.cpu().numpy(), want_ids), (mode, threads, cps)
                    assert np.array_equal(_host_u32(sc), want_sc), (mode, threads, cps)
        best, ms = ix.autotune(dq, dc, topk)
        assert ms > 0 and best.threads in (256, 512, 1024)
        ids, sc = ix.query(dq, dc, topk)   # the tuned default
        ix.sync()
        assert np.array_equal(ids.cpu().numpy(), want_ids)
        assert np.array_equal(_host_u32(sc), want_sc)


def test_uneven_queries_bit_exact():
    """The `uneven` mix: 30% planted, 70% random lognormal-nnz rows up to 2000."""
    from datagen.workloads import UNEVEN as w
    s = _slash()
    g = datagen.Generator()
    offs, cols = g.rows(w.seed, 0, w.n_rows)
    qo, qc, _ = g.queries(w.seed, w.qseed, 20_000, w.n_rows, **w.query_kwargs())
    assert np.diff(qo).max() > 1000
    p = s.Params(**w.params())
    want_ids, want_sc = _oracle_index(p, offs, cols).query(qo, qc, w.topk)
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        for mode in ("fused", "plain", "warp_fused", "warp_plain"):
            ids, sc = ix.query(_dev(qo), _dev(qc), w.topk, mode=mode)
            ix.sync()
            assert np.array_equal(ids.cpu().numpy(), want_ids), mode
            assert np.array_equal(_host_u32(sc), want_sc), mode


@pytest.mark.parametrize("sigma", ["0", "0.5", "3"])
def test_insert_filter_and_exact_fallback_bit_exact(sigma, monkeypatch):
    """The staging filter keeps ~R + sigma*sqrt(R) of a heavy bucket's new ids and
    proves in the merge that nothing below the R-th priority was dropped; with a
    small sigma that proof often fails (or the staging overflows) and the
    bucket takes the exact fallback.  Every sigma gives the oracle's index."""
    monkeypatch.setenv("SLASH_FILTER_SIGMA", sigma)
    s = _slash()
    g = datagen.Generator()
    n = 40_000
    offs, cols = g.rows(14, 0, n)
    p = s.Params(K=4, L=16, log2_buckets=5, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=14)
    want_slots, want_fill = _oracle_index(p, offs, cols).export()
    with s.Index(p) as ix:
        _gpu_insert(ix, offs, cols, [0, 3000, 3001, 25_000, n])
        ix.sync()
        slots, fill = ix.export()
    assert np.array_equal(fill, want_fill) and np.array_equal(slots, want_slots)


def test_streamed_device_rows_top100_bit_exact():
    """The `stream` shape scaled down: K=8, L=32, R=256, rows generated on the
    device chunk by chunk and inserted without being stored; top-100 queries."""
    from datagen.workloads import STREAM as w
    s = _slash()
    g = datagen.Generator()
    dg = datagen.DeviceRows(g)
    n, chunk = 200_000, 60_000
    p = s.Params(**w.params(capacity=n, log2_buckets=12))
    with s.Index(p) as ix:
        for r0 in range(0, n, chunk):
            o, c = dg.rows(w.seed, r0, min(chunk, n - r0))
            ix.insert(o, c)
        offs, cols = g.rows(w.seed, 0, n)
        qo, qc, src = g.queries(w.seed, w.qseed, 400, n, **w.query_kwargs())
        ids, sc = ix.query(_dev(qo), _dev(qc), w.topk)
        ix.sync()
        slots, fill = ix.export()
    oix = _oracle_index(p, offs, cols)
    ws, wf = oix.export()
    assert np.array_equal(fill, wf) and np.array_equal(slots, ws)
    want_ids, want_sc = oix.query(qo, qc, w.topk)
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(_host_u32(sc), want_sc)
    assert np.mean((ids.cpu().numpy() == src[:, None]).any(axis=1)) > 0.9  # planted rows are found


def test_insert_from_host_memory_chunks_not_aligned_to_pieces(monkeypatch):
    """5M host rows in 3M-row chunks: the copy pieces (2^21 rows) restart at each
    chunk, so the second chunk's pieces straddle the first chunk's grid.  The
    host-fed index equals the device-fed one array for array, and sampled
    buckets equal the oracle's."""
    import oracle as orc
    monkeypatch.setenv("SLASH_INSERT_CHUNK_ROWS", "3000000")
    s = _slash()
    g = datagen.Generator()
    n = 5_000_000
    offs, cols = g.rows(18, 0, n)
    p = s.Params(K=4, L=16, log2_buckets=14, reservoir=16, cm_rows=4, cm_width=4096, capacity=n, seed=18)
    h_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
    h_cols = torch.from_numpy(cols.view(np.int32)).pin_memory()
    with s.Index(p) as ix:
        bad = h_offs.clone()
        bad[4_500_000] = bad[4_500_001] + 1                  # one decreasing step, deep in the array
        with pytest.raises(s.SlashError) as e:
            ix.insert_host(bad, h_cols)
        assert e.value.code == s.SLASH_EINVAL and ix.size == 0
        assert ix.insert_host(h_offs, h_cols) == 0
        ix.sync()
        h_slots, h_fill = ix.export()
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        ix.sync()
        d_slots, d_fill = ix.export()
    assert np.array_equal(h_fill, d_fill) and np.array_equal(h_slots, d_slots)
    rng = np.random.default_rng(18)
    rt = rng.integers(0, p.L, 1500).astype(np.uint32)
    rb = rng.integers(0, 1 << p.log2_buckets, 1500).astype(np.uint32)
    oix = orc.Index(K=4, L=16, log2_buckets=14, reservoir=16, cm_rows=4, cm_width=4096, seed=18, capacity=n,
                    partial=(rt, rb))
    oix.insert(offs, cols, threads=datagen.default_threads())
    fill2 = h_fill.reshape(p.L, 1 << p.log2_buckets)
    slots2 = h_slots.reshape(p.L, 1 << p.log2_buckets, p.reservoir)
    for t, b in zip(rt, rb):
        want, wf = oix.bucket(int(t), int(b))
        assert fill2[t, b] == wf and np.array_equal(slots2[t, b], want), (int(t), int(b))


@pytest.mark.parametrize("chunk_rows", ["7000", "0"])
def test_insert_from_host_memory_bit_exact(chunk_rows, monkeypatch):
    """slash_insert_host (pinned host CSR, copies overlapped with hashing, many
    pieces and chunks) builds the same index as the device-fed insert and the oracle."""
    if chunk_rows != "0":
        monkeypatch.setenv("SLASH_INSERT_CHUNK_ROWS", chunk_rows)
    s = _slash()
    g = datagen.Generator()
    n = 50_000
    offs, cols = g.rows(16, 0, n)
    p = s.Params(K=6, L=64, log2_buckets=9, reservoir=16, cm_rows=4, cm_width=4096, capacity=n, seed=16)
    want_slots, want_fill = _oracle_index(p, offs, cols).export()
    h_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
    h_cols = torch.from_numpy(cols.view(np.int32)).pin_memory()
    with s.Index(p) as ix:
        assert ix.insert_host(h_offs[:20_001], h_cols) == 0
        assert ix.insert_host(h_offs[20_000:], h_cols) == 20_000
        ix.sync()
        slots, fill = ix.export()
    assert np.array_equal(fill, want_fill) and np.array_equal(slots, want_slots)

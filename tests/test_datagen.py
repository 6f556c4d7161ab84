"""The seeded input generator: determinism, shape of the distributions."""
import math

import numpy as np

import datagen


def test_rows_deterministic_and_thread_independent():
    g = datagen.Generator()
    a = g.rows(7, 100, 5000, threads=1)
    b = g.rows(7, 100, 5000, threads=6)
    c = g.rows(7, 0, 5100, threads=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # rows are keyed by their absolute index: a window equals the slice
    o = c[0][100:] - c[0][100]
    assert np.array_equal(o, a[0]) and np.array_equal(c[1][int(c[0][100]):], a[1])
    d = g.rows(8, 100, 5000)
    assert not np.array_equal(a[1][:1000], d[1][:1000])


def test_rows_shape():
    g = datagen.Generator()
    offs, cols = g.rows(0, 0, 50_000)
    nnz = np.diff(offs).astype(np.int64)
    assert nnz.min() >= 5 and nnz.max() <= 200
    assert abs(nnz.mean() - 40) < 0.2 and abs(nnz.var() - 40) < 2.0   # Poisson(40)
    assert cols.max() < (1 << 20)
    for i in range(0, 50_000, 997):
        r = cols[offs[i]:offs[i + 1]]
        assert np.all(np.diff(r.astype(np.int64)) > 0)  # strictly ascending: distinct
    # Zipf(1.1) head: the most popular feature is drawn with p1 = 1/H(2^20, 1.1)
    h = sum(k ** -1.1 for k in range(1, (1 << 20) + 1))
    p1 = 1 / h
    vals, cnt = np.unique(cols, return_counts=True)
    top = cnt.max() / len(nnz)
    expect = 1 - (1 - p1) ** 40  # present in a row of 40 draws (approximately)
    assert abs(top - expect) < 0.02


def test_planted_queries_keep_nnz_and_jaccard():
    g = datagen.Generator()
    n = 20_000
    offs, cols = g.rows(0, 0, n)
    qo, qc, src = g.queries(0, 3, 2000, n, p_perturb=0.2)
    assert np.all(src >= 0) and src.max() < n
    js = []
    for i in range(2000):
        q = set(qc[qo[i]:qo[i + 1]].tolist())
        r = set(cols[offs[src[i]]:offs[src[i] + 1]].tolist())
        assert len(q) == len(r) == qo[i + 1] - qo[i]
        js.append(len(q & r) / len(q | r))
    # E[(1-p)/(1+p)] = 0.667 for p = 0.2
    assert abs(np.mean(js) - (0.8 / 1.2)) < 0.02


def test_uneven_queries_mix():
    g = datagen.Generator()
    qo, qc, src = g.queries(0, 4, 20_000, 1000, planted_frac=0.3, p_perturb=0.2, rlo=1, rhi=2000)
    assert abs((src >= 0).mean() - 0.3) < 0.02
    nnz = np.diff(qo)[src < 0].astype(np.float64)
    assert nnz.min() >= 1 and nnz.max() <= 2000
    # lognormal(ln 40, 1): median 40
    assert abs(np.median(nnz) - 40) < 3
    assert abs(np.mean(np.log(nnz)) - math.log(40)) < 0.05


import pytest  # noqa: E402


@pytest.mark.gpu
def test_device_rows_match_host_rows():
    """The CUDA twin writes the host generator's bytes (streamed workloads)."""
    import torch
    g = datagen.Generator()
    dg = datagen.DeviceRows(g)
    for row0, n, lo, hi in [(0, 50_000, 5, 200), (123_456_789, 20_000, 5, 200), (7, 3000, 1, 2000)]:
        offs, cols = g.rows(11, row0, n, lo=lo, hi=hi)
        doffs, dcols = dg.rows(11, row0, n, lo=lo, hi=hi)
        torch.cuda.synchronize()
        assert np.array_equal(doffs.cpu().numpy().view(np.uint64), offs)
        assert np.array_equal(dcols.cpu().numpy().view(np.uint32), cols)

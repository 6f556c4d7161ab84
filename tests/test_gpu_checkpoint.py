"""Index checkpoints: a saved and reloaded index continues exactly like the
original (buckets, ids and query results), for both bucket kinds; damaged
files are refused."""
import os

import numpy as np
import pytest

import datagen
from test_gpu_parity import _dev

pytestmark = pytest.mark.gpu


def _s():
    import paper_2008_03260_b300 as s
    return s


def _data(n=20_000, nq=300):
    g = datagen.Generator()
    offs, cols = g.rows(5, 0, n)
    qo, qc, _ = g.queries(5, 2, nq, n)
    return offs, cols, qo, qc


def _damage(path, tmp_path):
    raw = open(path, "rb").read()
    bad = tmp_path / "flipped.ix"
    b = bytearray(raw)
    b[len(b) // 2] ^= 0x40
    bad.write_bytes(bytes(b))
    short = tmp_path / "short.ix"
    short.write_bytes(raw[:-8])
    longer = tmp_path / "long.ix"
    longer.write_bytes(raw + b"\0" * 8)
    return [bad, short, longer]


def test_reservoir_checkpoint_resumes_exactly(tmp_path):
    s = _s()
    offs, cols, qo, qc = _data()
    p = s.Params(K=4, L=16, log2_buckets=10, reservoir=16, shards=2, seed=3, capacity=20_000)
    half = 9_001
    with s.Index(p) as full:
        full.insert(_dev(offs), _dev(cols))
        want_slots, want_fill = full.export()
        want = [t.cpu().numpy() for t in full.query(_dev(qo), _dev(qc), 10)]
    path = str(tmp_path / "a.ix")
    with s.Index(p) as a:
        a.insert(_dev(offs[:half + 1]), _dev(cols))
        a.save(path)
    with s.Index.load(path) as b:
        assert b.p == p and b.size == half
        assert b.insert(_dev(offs[half:]), _dev(cols)) == half
        slots, fill = b.export()
        assert np.array_equal(slots, want_slots) and np.array_equal(fill, want_fill)
        got = [t.cpu().numpy() for t in b.query(_dev(qo), _dev(qc), 10)]
        assert all(np.array_equal(x, y) for x, y in zip(got, want))
    for bad in _damage(path, tmp_path):
        with pytest.raises(s.SlashError) as e:
            s.Index.load(str(bad))
        assert e.value.code == s.SLASH_EINVAL
    with pytest.raises(s.SlashError) as e:
        s.TkIndex.load(path)  # a reservoir checkpoint is not a sketch checkpoint
    assert e.value.code == s.SLASH_EINVAL


def test_sketch_checkpoint_resumes_exactly(tmp_path):
    s = _s()
    offs, cols, qo, qc = _data()
    p = s.TkParams(K=4, L=16, log2_buckets=9, rows=4, cells=32, shards=3, seed=9, capacity=20_000)
    with s.TkIndex(p) as full:
        full.insert(_dev(offs), _dev(cols))
        want_cells = full.export()
        want = [t.cpu().numpy() for t in full.query(_dev(qo), _dev(qc), 10)]
    path = str(tmp_path / "t.ix")
    with s.TkIndex(p) as a:
        a.insert(_dev(offs[:12_346]), _dev(cols))
        a.save(path)
    with s.TkIndex.load(path) as b:
        assert b.p == p and b.size == 12_345
        b.insert(_dev(offs[12_345:]), _dev(cols))
        assert np.array_equal(b.export(), want_cells)
        got = [t.cpu().numpy() for t in b.query(_dev(qo), _dev(qc), 10)]
        assert all(np.array_equal(x, y) for x, y in zip(got, want))
    for bad in _damage(path, tmp_path):
        with pytest.raises(s.SlashError) as e:
            s.TkIndex.load(str(bad))
        assert e.value.code == s.SLASH_EINVAL

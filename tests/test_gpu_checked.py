"""The checked build (libslash_checked.so, -DSLASH_CHECKS): every bucket key
and staging offset its kernels derive from the data is tested before use.
Insert (filters and the exact fallback), every query engine, shards and the
exchange run under it without raising the out-of-range flag, with results
equal to the oracle's.  Runs in a child process, which loads the checked
library instead of the service one."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import datagen, oracle
import paper_2008_03260_b300 as s
from paper_2008_03260_b300.multi import GpuPart, exchange_query_loopback, partition
assert s.library_path().endswith("libslash_checked.so")
checked, err = s.slash_debug_bounds()
assert checked and err == 0
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64 if a.dtype == np.uint64 else np.int32)).cuda()
g = datagen.Generator()
n = 40_000
offs, cols = g.rows(61, 0, n)
qo, qc, _ = g.queries(61, 62, 400, n, planted_frac=0.5, p_perturb=0.2)
for shards, R, B in ((1, 32, 8), (2, 16, 7)):
    kw = dict(K=4, L=16, log2_buckets=B, reservoir=R, cm_rows=4, cm_width=4096, shards=shards, seed=61, capacity=n)
    oix = oracle.Index(**kw)
    oix.insert(offs, cols)
    ws, wf = oix.export()
    with s.Index(s.Params(**kw)) as ix:
        ix.insert(dev(offs[:15001]), dev(cols))
        o2 = offs[15000:]
        ix.insert(dev(o2 - o2[0]), dev(cols[int(o2[0]):]))
        ix.sync()
        slots, fill = ix.export()
        assert np.array_equal(fill, wf) and np.array_equal(slots, ws), ("insert", shards)
        for mode in ("fused", "plain", "warp_fused", "warp_plain"):
            for k in (10, 25):
                if mode.startswith("warp") and k > 10:
                    continue
                ids, sc = ix.query(dev(qo), dev(qc), k, mode=mode)
                ix.sync()
                want_ids, want_sc = oix.query(qo, qc, k)
                assert np.array_equal(ids.cpu().numpy(), want_ids), (mode, k, shards)
                assert np.array_equal(sc.cpu().numpy().view(np.uint32), want_sc), (mode, k, shards)
    assert s.slash_debug_bounds() == (True, 0), shards
# the exchange's kernels
parts, ixs = [], []
kw = dict(K=4, L=16, log2_buckets=8, reservoir=32, cm_rows=4, cm_width=4096, seed=61, capacity=n)
for r in range(2):
    lo, cnt = partition(r, 2, n)
    ix = s.Index(s.Params(**kw))
    ix.set_next_id(lo)
    o = offs[lo:lo + cnt + 1]
    ix.insert(dev(o - o[0]), dev(cols[int(o[0]):int(o[-1])]))
    ixs.append(ix)
    parts.append(GpuPart(ix))
ids, sc = exchange_query_loopback(parts, dev(qo), dev(qc), 10, chunk=128)
torch.cuda.synchronize()
oix = oracle.Index(**kw, shards=2)
oix.insert(offs, cols)
want_ids, want_sc = oix.query(qo, qc, 10)
assert np.array_equal(ids.cpu().numpy(), want_ids) and np.array_equal(sc.cpu().numpy().view(np.uint32), want_sc)
for ix in ixs:
    ix.sync()
    ix.close()
assert s.slash_debug_bounds() == (True, 0)
print("checked build: no index out of range")
'''


def test_checked_build_finds_no_index_out_of_range():
    env = dict(os.environ, SLASH_CHECKED="1", SLASH_FILTER_SIGMA="0")  # sigma 0: the exact fallback runs often
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no index out of range" in r.stdout


def test_service_build_reports_unchecked():
    import paper_2008_03260_b300 as s
    if os.environ.get("SLASH_CHECKED") == "1":
        pytest.skip("this process loaded the checked build")
    assert s.slash_debug_bounds() == (False, 0)

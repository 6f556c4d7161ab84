"""The allocation-free query entry point (collected last on purpose).

slash_query_static serves callers that cannot allocate device memory when they
query (hosts with pre-sized memory pools): its scratch is a fixed
array inside the library.  Called through the C ABI, it must give exactly the
plain query path's results, on consecutive calls that reuse that array.
"""
import ctypes

import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.view(np.int64 if a.dtype == np.uint64 else np.int32))).cuda()


def _static(s, ix, qo, qc, k):
    import torch
    nq = qo.numel() - 1
    ids = torch.full((nq, k), 7, dtype=torch.int32, device="cuda")
    sc = torch.full((nq, k), 7, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = s._lib.slash_query_static(ix.h, qo.data_ptr(), qc.data_ptr(), nq, k, ids.data_ptr(), sc.data_ptr(),
                                   ctypes.c_void_p(st or None))
    return rc, ids, sc


def test_static_scratch_query_equals_plain_query_twice():
    import torch

    import paper_2008_03260_b300 as s
    g = datagen.Generator()
    n = 20_000
    offs, cols = g.rows(21, 0, n)
    p = s.Params(K=4, L=16, log2_buckets=10, reservoir=32, cm_rows=4, cm_width=4096, shards=2, capacity=n, seed=21)
    with s.Index(p) as ix:
        ix.insert(_dev(offs), _dev(cols))
        for call, (qseed, nq, k) in enumerate([(1, 3000, 10), (2, 1700, 25)]):
            qo, qc, _ = g.queries(21, qseed, nq, n, planted_frac=0.3, p_perturb=0.2)
            dqo, dqc = _dev(qo), _dev(qc)
            rc, ids, sc = _static(s, ix, dqo, dqc, k)
            assert rc == s.SLASH_OK, (call, s.slash_strerror(rc))
            want_ids, want_sc = ix.query(dqo, dqc, k, mode="plain", threads=512)
            torch.cuda.synchronize()
            assert s.slash_sync(ix.h) == s.SLASH_OK
            assert torch.equal(ids, want_ids), call
            assert torch.equal(sc, want_sc), call
        # beyond the fixed scratch: rejected before any launch, outputs untouched
        big = np.zeros((1 << 22) // 16 + 2, np.uint64)
        rc, ids, _ = _static(s, ix, _dev(big), _dev(np.zeros(1, np.uint32)), 10)
        assert rc == s.SLASH_EINVAL
        torch.cuda.synchronize()
        assert int(ids.min()) == 7 and int(ids.max()) == 7

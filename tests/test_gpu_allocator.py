"""The allocator hook: the index's workspace comes from the caller's allocator
(here PyTorch's caching allocator, counted), results stay the oracle's, every
allocation is released, and an allocator with no memory makes the call fail
with SLASH_ENOMEM and the index unchanged."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    a = a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class Counted:
    """PyTorch's caching allocator, with a record of what the library took."""

    def __init__(self):
        import paper_2008_03260_b300 as s
        self.alloc_, self.release_ = s.torch_allocator()
        self.live, self.allocs, self.frees = {}, 0, 0

    def alloc(self, n):
        p = self.alloc_(n)
        self.live[p] = n
        self.allocs += 1
        return p

    def release(self, p):
        assert p in self.live, "released a pointer the allocator did not give"
        del self.live[p]
        self.frees += 1
        self.release_(p)


def test_workspace_from_the_torch_allocator_equals_oracle():
    import paper_2008_03260_b300 as s
    g = datagen.Generator()
    n = 20_000
    offs, cols = g.rows(41, 0, n)
    qo, qc, _ = g.queries(41, 42, 500, n)
    p = s.Params(K=4, L=16, log2_buckets=11, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=41)
    a = Counted()
    ix = s.Index(p)
    ix.set_allocator(a.alloc, a.release)
    before = torch.cuda.memory_allocated()
    ix.insert(_dev(offs[:5001]), _dev(cols))                                 # insert workspace
    h_offs = torch.from_numpy((offs[5000:] - offs[5000]).view(np.int64)).pin_memory()
    h_cols = torch.from_numpy(cols[int(offs[5000]):].view(np.int32)).pin_memory()
    assert ix.insert_host(h_offs, h_cols) == 5000                            # + host staging, larger insert
    ids, sc = ix.query(_dev(qo), _dev(qc), 10, mode="plain")                 # + plain-query addresses
    ix.sync()
    held = sum(a.live.values())
    assert a.allocs >= 3 and held > 0
    assert torch.cuda.memory_allocated() - before >= held                    # the caller's allocator holds it
    slots, fill = ix.export()
    ix.close()
    assert not a.live and a.frees == a.allocs                                # every piece went back
    oix = oracle.Index(K=4, L=16, log2_buckets=11, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=41)
    oix.insert(offs, cols)
    ws, wf = oix.export()
    assert np.array_equal(fill, wf) and np.array_equal(slots, ws)
    want_ids, want_sc = oix.query(qo, qc, 10)
    assert np.array_equal(ids.cpu().numpy(), want_ids)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), want_sc)


def test_allocator_without_memory_fails_cleanly_and_can_be_replaced():
    import paper_2008_03260_b300 as s
    g = datagen.Generator()
    n = 8_000
    offs, cols = g.rows(43, 0, n)
    p = s.Params(K=4, L=16, log2_buckets=10, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=43)
    d_cols = _dev(cols)
    with s.Index(p) as ix:
        ix.insert(_dev(offs[:2001]), d_cols)                                 # cudaMalloc workspace
        ix.sync()
        slots0, fill0 = ix.export()
        ix.set_allocator(lambda nbytes: None, lambda ptr: None)              # releases that workspace
        with pytest.raises(s.SlashError) as e:
            ix.insert(_dev(offs[2000:]), d_cols)
        assert e.value.code == s.SLASH_ENOMEM
        assert ix.size == 2000
        slots1, fill1 = ix.export()
        assert np.array_equal(slots0, slots1) and np.array_equal(fill0, fill1)
        ix.set_allocator()                                                   # back to cudaMalloc
        assert ix.insert(_dev(offs[2000:]), d_cols) == 2000
        ix.sync()
        slots, fill = ix.export()
    oix = oracle.Index(K=4, L=16, log2_buckets=10, reservoir=32, cm_rows=4, cm_width=4096, capacity=n, seed=43)
    oix.insert(offs, cols)
    ws, wf = oix.export()
    assert np.array_equal(fill, wf) and np.array_equal(slots, ws)

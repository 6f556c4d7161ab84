"""Serving loop: admission/batching host logic on CPU (fake executor), and the
GPU loop's results equal to each request answered alone (tolerance zero)."""
import dataclasses
import time

import numpy as np
import pytest

import datagen


class FakeExecutor:
    """Answers query i of a batch with (nnz, first col, ...) after a fixed delay."""

    def __init__(self, topk, delay=0.002):
        self.topk, self.delay = topk, delay
        self.launched = []
        self.peak_inflight = 0
        self.live = 0

    def launch(self, slot, offs, cols):
        nq = len(offs) - 1
        ids = np.full((nq, self.topk), -1, np.int32)
        for q in range(nq):
            row = cols[int(offs[q]):int(offs[q + 1])]
            ids[q, 0] = len(row)
            if len(row):
                ids[q, 1] = row[0]
        self.launched.append(nq)
        self.live += 1
        self.peak_inflight = max(self.peak_inflight, self.live)
        return [time.perf_counter() + self.delay, ids, False]

    def done(self, h):
        return time.perf_counter() >= h[0]

    def collect(self, h):
        self.live -= 1
        return h[1], np.zeros_like(h[1], dtype=np.uint32), h[0]


def _pool(n=3000):
    g = datagen.Generator()
    qo, qc, _ = g.queries(0, 2, n, 1000, planted_frac=0.3, p_perturb=0.2)
    return qo, qc


def test_batcher_admission_respects_budget_and_order():
    from paper_2008_03260_b300.serve import Batcher, Request, request_bytes
    qo, qc = _pool(200)
    reqs = []
    for i in range(20):
        o = qo[i * 10:i * 10 + 11]
        reqs.append(Request(i, (o - o[0]).astype(np.uint64), qc[int(o[0]):int(o[-1])], 0.0))
    budget = sum(request_bytes(r, 10) for r in reqs[:5])
    b = Batcher(slots=3, topk=10, mem_budget=budget, max_batch_queries=30)
    for r in reqs:
        b.arrive(r)
    first = b.next_batch(0)
    assert [r.rid for r in first.reqs] == [0, 1, 2]          # capped at 30 queries
    second = b.next_batch(1)
    assert [r.rid for r in second.reqs] == [3, 4]             # capped by the memory budget
    assert b.next_batch(2) is None and b.mem_in_use <= budget
    b.finish(0)
    third = b.next_batch(0)
    got = [r.rid for r in third.reqs]
    assert got == list(range(5, 5 + len(got))) and got         # arrival order kept
    nxt = reqs[5 + len(got)]                                   # the next one did not fit
    assert b.mem_in_use + request_bytes(nxt, 10) > budget or sum(r.nq for r in third.reqs) + nxt.nq > 30
    assert b.mem_in_use <= budget
    huge = Request(99, np.array([0, 1], np.uint64), np.zeros(1, np.uint32), 0.0)
    tiny = Batcher(slots=1, topk=10, mem_budget=8, max_batch_queries=30)
    tiny.arrive(huge)
    assert tiny.refused == [huge] and not tiny.queue


def test_serve_loop_slices_results_per_request():
    from paper_2008_03260_b300.serve import poisson_requests, serve
    qo, qc = _pool()
    reqs = poisson_requests(20_000.0, 300, qo, qc, seed=1, max_size=64)
    ex = FakeExecutor(topk=5)
    res, summ = serve(reqs, ex, topk=5, slots=3, mem_budget=1 << 20, max_batch_queries=256)
    assert summ["requests"] == 300 and summ["refused"] == 0
    assert ex.peak_inflight <= 3 and max(ex.launched) <= 256
    assert summ["batches"] < 300   # requests that queued up were batched together
    by = {r.rid: r for r in res}
    for q in reqs:
        r = by[q.rid]
        assert r.ids.shape == (q.nq, 5) and r.latency >= 0
        for i in range(q.nq):
            row = q.cols[int(q.offs[i]):int(q.offs[i + 1])]
            assert r.ids[i, 0] == len(row)
            if len(row):
                assert r.ids[i, 1] == row[0]


@pytest.mark.gpu
def test_gpu_serving_results_equal_alone():
    """Requests mixed into overlapping batches on several streams get exactly the
    answer they get when queried alone (and the oracle's, for a sample)."""
    import torch

    import oracle
    import paper_2008_03260_b300 as s
    from paper_2008_03260_b300.serve import GpuExecutor, poisson_requests, serve
    g = datagen.Generator()
    n = 30_000
    offs, cols = g.rows(0, 0, n)
    qo, qc, _ = g.queries(0, 3, 20_000, n, planted_frac=0.3, p_perturb=0.2)
    p = s.Params(K=4, L=16, log2_buckets=12, reservoir=32, cm_rows=4, cm_width=8192, shards=8, capacity=n)
    dev = lambda a: torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32)).cuda()
    with s.Index(p) as ix:
        ix.insert(dev(offs), dev(cols))
        ix.sync()
        reqs = poisson_requests(50_000.0, 400, qo, qc, seed=5, max_size=512)
        ex = GpuExecutor(ix, topk=10, slots=4)
        res, summ = serve(reqs, ex, topk=10, slots=4, mem_budget=64 << 20, max_batch_queries=2048)
        assert summ["requests"] == 400 and summ["batches"] < 400
        by = {r.rid: r for r in res}
        for q in reqs:
            ids, sc = ix.query(dev(q.offs), dev(q.cols), 10, mode="fused")
            assert np.array_equal(by[q.rid].ids, ids.cpu().numpy()), q.rid
            assert np.array_equal(by[q.rid].scores, sc.cpu().numpy().view(np.uint32)), q.rid
        ix.sync()
    oix = oracle.Index(K=4, L=16, log2_buckets=12, reservoir=32, cm_rows=4, cm_width=8192, shards=8,
                       capacity=n)
    oix.insert(offs, cols)
    for q in reqs[:40]:
        want_ids, want_sc = oix.query(q.offs, q.cols, 10)
        assert np.array_equal(by[q.rid].ids, want_ids) and np.array_equal(by[q.rid].scores, want_sc)


def test_queued_requests_past_their_deadline_are_cancelled():
    """A deadline that passes while the request waits in the queue cancels it
    (SLASH_ETIMEOUT, no result); the others are answered as usual."""
    from paper_2008_03260_b300.serve import SLASH_ETIMEOUT, Request, serve
    qo, qc = _pool(40)
    reqs = []
    for i in range(12):
        o = qo[i * 3:i * 3 + 4]
        dl = 0.005 if i % 3 == 2 else float("inf")     # a third must start within 5 ms
        reqs.append(Request(i, (o - o[0]).astype(np.uint64), qc[int(o[0]):int(o[-1])], 0.0, dl))
    ex = FakeExecutor(topk=4, delay=0.05)                # one slot, 50 ms per batch
    res, summ = serve(reqs, ex, topk=4, slots=1, mem_budget=1 << 20, max_batch_queries=3)
    by = {r.rid: r for r in res}
    assert by[0].status == 0 and by[0].ids is not None   # launched at once
    late = [i for i in range(12) if i % 3 == 2 and i > 0]
    assert all(by[i].status == SLASH_ETIMEOUT and by[i].ids is None for i in late)
    assert all(by[i].status == 0 for i in range(12) if i not in late)
    assert summ["cancelled"] == len(late) and summ["requests"] == 12 - len(late)
    assert summ["p99_queued_ms"] >= 0 and summ["p99_device_ms"] >= 0


def test_native_serve_validates_before_touching_the_gpu():
    """slash_serve checks its options and arrays before any CUDA call (the
    index handle is never dereferenced on these paths)."""
    import ctypes

    import paper_2008_03260_b300 as s
    fake = ctypes.c_void_p(1)
    arr = np.array([0.0, 0.1], dtype=np.float64)
    rq = np.array([0, 1, 2], dtype=np.uint64)
    offs = np.array([0, 2, 3], dtype=np.uint64)
    cols = np.array([1, 2, 3], dtype=np.uint32)
    out = [np.empty(20, np.int32), np.empty(20, np.uint32), np.empty(2), np.empty(2), np.empty(2, np.int32)]

    def call(o, arrival=arr, req_q=rq, offsets=offs, n=2):
        return s._lib.slash_serve(fake, ctypes.byref(o), n, arrival.ctypes.data, req_q.ctypes.data,
                                  offsets.ctypes.data, cols.ctypes.data, *[a.ctypes.data for a in out], None)

    ok = dict(slots=2, max_batch_queries=8, topk=10, mode=s.SLASH_QUERY_FUSED, threads=0, reserve_sms=0,
              small_queries=0, flags=0, timeout_s=0.0)
    for bad in (dict(slots=0), dict(slots=17), dict(max_batch_queries=0), dict(topk=0), dict(topk=257),
                dict(mode=s.SLASH_QUERY_PLAIN), dict(mode=s.SLASH_QUERY_WARP_PLAIN), dict(flags=2),
                dict(reserve_sms=8)):  # an SM reserve needs a small-batch size
        assert call(s.slash_serve_opts(**{**ok, **bad})) == s.SLASH_EINVAL, bad
    o = s.slash_serve_opts(**ok)
    assert call(o, arrival=np.array([0.2, 0.1])) == s.SLASH_EINVAL            # arrivals go back in time
    assert call(o, arrival=np.array([-1.0, 0.1])) == s.SLASH_EINVAL
    assert call(o, req_q=np.array([1, 1, 2], dtype=np.uint64)) == s.SLASH_EINVAL  # must start at query 0
    assert call(o, req_q=np.array([0, 2, 1], dtype=np.uint64)) == s.SLASH_EINVAL
    assert call(o, offsets=np.array([0, 3, 2], dtype=np.uint64)) == s.SLASH_EINVAL
    assert call(o, n=0) == s.SLASH_OK                                             # nothing to serve


@pytest.mark.gpu
def test_native_serving_equals_oracle_refuses_and_cancels():
    """The native loop's answers equal the oracle's for every answered request;
    requests larger than a batch are refused; a deadline that has always passed
    cancels every request."""
    import torch

    import oracle
    import paper_2008_03260_b300 as s
    from paper_2008_03260_b300.serve import SLASH_EBUSY, SLASH_ETIMEOUT, poisson_requests, serve_native
    g = datagen.Generator()
    n = 30_000
    offs, cols = g.rows(0, 0, n)
    qo, qc, _ = g.queries(0, 3, 20_000, n, planted_frac=0.3, p_perturb=0.2)
    p = s.Params(K=4, L=16, log2_buckets=12, reservoir=32, cm_rows=4, cm_width=8192, shards=8, capacity=n)
    dev = lambda a: torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32)).cuda()
    oix = oracle.Index(K=4, L=16, log2_buckets=12, reservoir=32, cm_rows=4, cm_width=8192, shards=8,
                       capacity=n)
    oix.insert(offs, cols)
    with s.Index(p) as ix:
        ix.insert(dev(offs), dev(cols))
        ix.sync()
        reqs = poisson_requests(50_000.0, 400, qo, qc, seed=7, max_size=512)
        want = {q.rid: oix.query(q.offs, q.cols, 10) for q in reqs if q.nq <= 300}
        # (schedule, SMs left to small batches, small-batch size, caller arrays page-locked):
        # one priority for all, then high-priority small batches beside large ones held to
        # 48 and to 8 SMs; and every batch through the slots' buffers
        for mode, reserve, small, pin in (("fused", 0, 0, True), ("warp_fused", 0, 0, True),
                                          ("fused", 100, 32, True), ("warp_fused", 140, 64, True),
                                          ("fused", 0, 0, False)):
            res, summ = serve_native(reqs, ix, topk=10, slots=4, max_batch_queries=300, mode=mode,
                                     reserve_sms=reserve, small_queries=small, pin=pin)
            by = {r.rid: r for r in res}
            big = [q for q in reqs if q.nq > 300]
            assert big and all(by[q.rid].status == SLASH_EBUSY for q in big)
            assert summ["refused"] == len(big) and summ["requests"] == len(reqs) - len(big)
            for q in reqs:
                r = by[q.rid]
                if q.nq > 300:
                    continue
                assert r.status == 0 and r.arrival <= r.launched <= r.done
                want_ids, want_sc = want[q.rid]
                assert np.array_equal(r.ids, want_ids), (mode, reserve, q.rid)
                assert np.array_equal(r.scores, want_sc), (mode, reserve, q.rid)
        # a device-memory budget of the median request's bytes: the larger requests are
        # refused, the rest answered as alone (one or two batches in flight at a time)
        from paper_2008_03260_b300.serve import request_bytes
        rb = {q.rid: request_bytes(q, 10) for q in reqs}
        budget = sorted(rb.values())[len(reqs) // 2]
        res, summ = serve_native(reqs, ix, topk=10, slots=4, max_batch_queries=300, mem_budget=budget)
        by = {r.rid: r for r in res}
        for q in reqs:
            r = by[q.rid]
            if q.nq > 300 or rb[q.rid] > budget:
                assert r.status == SLASH_EBUSY, q.rid
                continue
            assert r.status == 0 and np.array_equal(r.ids, want[q.rid][0]), q.rid
            assert np.array_equal(r.scores, want[q.rid][1]), q.rid
        assert summ["refused"] == sum(1 for q in reqs if q.nq > 300 or rb[q.rid] > budget)
        # a launch held to a few SMs answers as one over the whole GPU
        q1 = int(qo[2000])
        d_qo, d_qc = dev((qo[:2001] - qo[0]).astype(np.uint64)), dev(np.ascontiguousarray(qc[int(qo[0]):q1]))
        for mode in ("fused", "plain", "warp_fused", "warp_plain"):
            a_ids, a_sc = ix.query(d_qo, d_qc, 10, mode=mode)
            b_ids, b_sc = ix.query(d_qo, d_qc, 10, mode=mode, max_sms=3)
            assert torch.equal(a_ids, b_ids) and torch.equal(a_sc, b_sc), mode
        # every request arrives at time 0 and may wait 1 ns: by the loop's first look
        # (tens of ns after its start) every deadline has passed
        at0 = [dataclasses.replace(q, arrival=0.0) for q in reqs]
        res, summ = serve_native(at0, ix, topk=10, slots=2, max_batch_queries=4096, timeout_s=1e-9)
        assert all(r.status == SLASH_ETIMEOUT and r.ids is None for r in res)
        assert summ["cancelled"] == len(reqs)
        ix.sync()

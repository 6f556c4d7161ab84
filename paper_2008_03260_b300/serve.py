"""Serving loop: continuous batching of query requests against a resident index.

Requests (each a CSR batch of 1..4096 queries) arrive over time.  The loop
keeps the index resident on the device and runs up to ``slots`` batches at
once, each on its own CUDA stream, so batches overlap on the device.  Whenever
a slot finishes, the requests that arrived meanwhile are admitted in arrival
order into the next batch, as long as the batch stays under
``max_batch_queries`` and the device bytes of all in-flight batches (CSR
inputs + outputs) stay under ``mem_budget``.  A request that could never fit
is refused (``SLASH_EBUSY``).  A request may carry a deadline: if it is still
queued when its deadline passes it is cancelled (``SLASH_ETIMEOUT``, no
result) instead of launched.  Latency = answers in the caller's hands -
arrival, on the host's clock; each result also records when its batch was
launched and the batch's span on the device (CUDA timing events), so a
latency splits into time queued, host time and device time.

The batching logic (:class:`Batcher`) is host code with no device calls; the
device work is behind :class:`GpuExecutor`, which issues the fused query
kernel through the C ABI.  Results do not depend on how requests are grouped:
every query is answered by one CTA from the same read-only index.
:func:`serve_native` runs the same policy in the library's C++ loop
(``slash_serve``), which is the one the bench reports.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

SLASH_EBUSY = -5
SLASH_ETIMEOUT = -6


@dataclass
class Request:
    rid: int
    offs: np.ndarray          # uint64 [nq+1], offs[0] == 0
    cols: np.ndarray          # uint32 [nnz]
    arrival: float            # seconds since the start of the run
    deadline: float = math.inf  # cancel if not launched by then (seconds since the start)

    @property
    def nq(self) -> int:
        return len(self.offs) - 1


@dataclass
class Result:
    rid: int
    arrival: float
    launched: float = math.nan
    done: float = math.nan
    ids: np.ndarray | None = None
    scores: np.ndarray | None = None
    status: int = 0
    device: float = math.nan  # the batch's device span (copy in to copy back), seconds

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Batch:
    slot: int
    reqs: list
    nq: int
    nbytes: int
    handle: object = None
    launched: float = math.nan


def request_bytes(r: Request, topk: int) -> int:
    """Device bytes a request occupies while in flight: CSR in, ids + scores out."""
    return 8 * (r.nq + 1) + 4 * len(r.cols) + 8 * r.nq * topk


class Batcher:
    """Admission and batching, independent of the device."""

    def __init__(self, slots: int, topk: int, mem_budget: int, max_batch_queries: int):
        self.slots, self.topk = slots, topk
        self.mem_budget, self.max_batch = mem_budget, max_batch_queries
        self.queue: collections.deque[Request] = collections.deque()
        self.inflight: list[Batch | None] = [None] * slots
        self.mem_in_use = 0
        self.refused: list[Request] = []

    def arrive(self, r: Request) -> None:
        if request_bytes(r, self.topk) > self.mem_budget or r.nq > self.max_batch:
            self.refused.append(r)  # could never be admitted
        else:
            self.queue.append(r)

    def free_slots(self) -> list[int]:
        return [s for s, b in enumerate(self.inflight) if b is None]

    def expire(self, now: float) -> list[Request]:
        """Remove and return the queued requests whose deadline has passed."""
        if not any(r.deadline < now for r in self.queue):
            return []
        gone = [r for r in self.queue if r.deadline < now]
        self.queue = collections.deque(r for r in self.queue if r.deadline >= now)
        return gone

    def next_batch(self, slot: int) -> Batch | None:
        """Requests in arrival order while the batch and the memory budget allow."""
        reqs, nq, nb = [], 0, 0
        while self.queue:
            r = self.queue[0]
            rb = request_bytes(r, self.topk)
            if nq + r.nq > self.max_batch or self.mem_in_use + nb + rb > self.mem_budget:
                break
            reqs.append(self.queue.popleft())
            nq += r.nq
            nb += rb
        if not reqs:
            return None
        b = Batch(slot, reqs, nq, nb)
        self.inflight[slot] = b
        self.mem_in_use += nb
        return b

    def finish(self, slot: int) -> Batch:
        b = self.inflight[slot]
        self.inflight[slot] = None
        self.mem_in_use -= b.nbytes
        return b

    def busy(self) -> bool:
        return bool(self.queue) or any(b is not None for b in self.inflight)


def concat_csr(reqs: list[Request], offs_out: np.ndarray | None = None,
               cols_out: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """One CSR batch of the requests' queries (into the given buffers if any)."""
    nqs = [r.nq for r in reqs]
    nq, nnz = sum(nqs), sum(len(r.cols) for r in reqs)
    offs = np.zeros(nq + 1, dtype=np.uint64) if offs_out is None else offs_out[:nq + 1]
    cols = np.empty(nnz, dtype=np.uint32) if cols_out is None else cols_out[:nnz]
    offs[0] = 0
    pos, base = 0, 0
    for r in reqs:
        offs[pos + 1:pos + r.nq + 1] = r.offs[1:] + np.uint64(base)
        cols[base:base + len(r.cols)] = r.cols
        pos += r.nq
        base += len(r.cols)
    return offs, cols


class _SlotBuffers:
    """Page-locked host and device buffers of one slot.  A batch's offsets and
    features share one buffer (one copy to the device), its ids and scores
    another (one copy back).  Grown (doubling) only when a batch needs more:
    after warm-up no batch pins or allocates memory."""

    def __init__(self, torch, topk: int, queries: int, nnz: int):
        self.torch, self.topk = torch, topk
        self.in_cap = self.out_cap = 0
        self.ensure(queries, nnz)

    @staticmethod
    def _in_layout(queries: int, nnz: int) -> tuple[int, int]:
        """Byte offset of the features (16-byte aligned, after the offsets) and the input size."""
        c0 = (8 * (queries + 1) + 15) & ~15
        return c0, c0 + 4 * max(nnz, 1)

    def ensure(self, queries: int, nnz: int) -> None:
        torch = self.torch
        need = self._in_layout(queries, nnz)[1]
        if need > self.in_cap:
            self.in_cap = max(need, 2 * self.in_cap)
            self.h_in = torch.empty(self.in_cap, dtype=torch.uint8, pin_memory=True)
            self.d_in = torch.empty(self.in_cap, dtype=torch.uint8, device="cuda")
        need = 8 * max(queries, 1) * self.topk
        if need > self.out_cap:
            self.out_cap = max(need, 2 * self.out_cap)
            self.h_out = torch.empty(self.out_cap, dtype=torch.uint8, pin_memory=True)
            self.d_out = torch.empty(self.out_cap, dtype=torch.uint8, device="cuda")

    def views(self, nq: int, nnz: int):
        """(host offsets, host features, device offsets, device features, input bytes,
        device ids, device scores, output bytes) of an nq-query batch."""
        torch = self.torch
        c0, nin = self._in_layout(nq, nnz)
        ob = 4 * nq * self.topk
        return (self.h_in[:8 * (nq + 1)].view(torch.int64), self.h_in[c0:nin].view(torch.int32),
                self.d_in[:8 * (nq + 1)].view(torch.int64), self.d_in[c0:nin].view(torch.int32), nin,
                self.d_out[:ob].view(torch.int32).view(nq, self.topk),
                self.d_out[ob:2 * ob].view(torch.int32).view(nq, self.topk), 2 * ob)

    def results(self, nq: int) -> tuple[np.ndarray, np.ndarray]:
        ob = 4 * nq * self.topk
        h = self.h_out.numpy()
        return (h[:ob].view(np.int32).reshape(nq, self.topk).copy(),
                h[ob:2 * ob].view(np.uint32).reshape(nq, self.topk).copy())


class GpuExecutor:
    """One CUDA stream and one set of preallocated buffers per slot: the batch
    is written into the slot's page-locked buffers, copied to the device, queried
    and the results copied back, all on the slot's stream.  The query runs the
    given schedule (mode, threads), or the index's default one when mode is None
    (the schedule slash_autotune picked, if it ran)."""

    def __init__(self, ix, topk: int, slots: int, threads: int = 0, queries: int = 1 << 12, nnz: int = 1 << 18,
                 mode: str | None = "fused"):
        import torch
        self.torch = torch
        self.ix, self.topk, self.threads = ix, topk, threads
        self.sched = {} if mode is None else {"mode": mode, "threads": threads}
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.bufs = [_SlotBuffers(torch, topk, queries, nnz) for _ in range(slots)]
        self.ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(slots)]
        self.events = [torch.cuda.Event(enable_timing=True) for _ in range(slots)]

    def launch_reqs(self, slot: int, reqs: list[Request]):
        torch = self.torch
        st, b = self.streams[slot], self.bufs[slot]
        nq, nnz = sum(r.nq for r in reqs), sum(len(r.cols) for r in reqs)
        b.ensure(nq, nnz)
        h_offs, h_cols, d_offs, d_cols, nin, d_ids, d_sc, nout = b.views(nq, nnz)
        # the slot's previous batch has completed (the loop only reuses a free
        # slot), so its host buffers can be overwritten
        concat_csr(reqs, h_offs.numpy().view(np.uint64), h_cols.numpy().view(np.uint32))
        with torch.cuda.stream(st):
            self.ev0[slot].record(st)
            b.d_in[:nin].copy_(b.h_in[:nin], non_blocking=True)
            self.ix.query(d_offs, d_cols, self.topk, st, d_ids_out=d_ids, d_scores_out=d_sc, **self.sched)
            b.h_out[:nout].copy_(b.d_out[:nout], non_blocking=True)
            ev = self.events[slot]
            ev.record(st)
        return (ev, slot, nq)

    def launch(self, slot: int, offs: np.ndarray, cols: np.ndarray):
        """A batch given as one CSR array (offs[0] == 0)."""
        return self.launch_reqs(slot, [Request(-1, offs, cols, 0.0)])

    def done(self, h) -> bool:
        return h[0].query()

    def collect(self, h) -> tuple[np.ndarray, np.ndarray, float]:
        ev, slot, nq = h
        ev.synchronize()
        ids, sc = self.bufs[slot].results(nq)
        return ids, sc, time.perf_counter()  # the answers are in the caller's hands

    def device_span(self, h) -> float:
        """Seconds from the batch's copy in to the end of its copy back (completed batch)."""
        ev, slot, _ = h
        return self.ev0[slot].elapsed_time(ev) / 1e3


def summarize(requests: list[Request], res: dict, n_batches: int) -> dict:
    """Latency percentiles and throughput of a served request stream."""
    done = [r for r in res.values() if r.status == 0]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    nq = sum(q.nq for q in requests if res[q.rid].status == 0)
    span = max(r.done for r in done) - min(r.arrival for r in done) if done else 1.0
    p99 = float(np.percentile(lat, 99))
    size = {q.rid: q.nq for q in requests}
    small = np.array([r.latency for r in done if size[r.rid] <= 64])
    tail = [r for r in done if r.latency >= p99] or done
    return {"requests": len(done),
            "refused": sum(1 for r in res.values() if r.status == SLASH_EBUSY),
            "cancelled": sum(1 for r in res.values() if r.status == SLASH_ETIMEOUT),
            "queries": nq, "batches": n_batches,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * p99,
            "mean_ms": 1e3 * float(lat.mean()), "queries_per_s": nq / span if span > 0 else float("nan"),
            "span_s": span,
            # where the slowest 1% spent their time: queued before launch, from
            # launch to answers in hand, and of that the batch's span on the device
            "p99_queued_ms": 1e3 * float(np.mean([r.launched - r.arrival for r in tail])) if tail else 0.0,
            "p99_device_ms": 1e3 * float(np.mean([r.done - r.launched for r in tail])) if tail else 0.0,
            "p99_gpu_span_ms": 1e3 * float(np.nanmean([r.device for r in tail]))
            if tail and not all(math.isnan(r.device) for r in tail) else float("nan"),
            # the tail of small requests alone (sizes are log-uniform: the slowest 1%
            # overall are mostly the largest requests)
            "p50_small_ms": 1e3 * float(np.percentile(small, 50)) if len(small) else 0.0,
            "p99_small_ms": 1e3 * float(np.percentile(small, 99)) if len(small) else 0.0}


def serve_native(requests: list[Request], ix, *, topk: int, slots: int = 4, max_batch_queries: int = 8192,
                 mode: str = "fused", threads: int = 0, timeout_s: float = 0.0, reserve_sms: int = 0,
                 small_queries: int = 0, pin: bool = True, mem_budget: int = 16 << 30
                 ) -> tuple[list[Result], dict]:
    """The same request stream through the library's native loop (slash_serve):
    admission, batching and the slots' streams run in C++; this function only
    lays the requests out as arrays and reads the answers back."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    arrival = np.array([r.arrival for r in reqs], dtype=np.float64)
    req_q = np.zeros(len(reqs) + 1, dtype=np.uint64)
    np.cumsum([r.nq for r in reqs], out=req_q[1:])
    offs, cols = concat_csr(reqs)
    ids, sc, launched, done, status, device = ix.serve(arrival, req_q, offs, cols, topk, slots=slots,
                                               max_batch_queries=max_batch_queries, mode=mode, threads=threads,
                                               timeout_s=timeout_s, reserve_sms=reserve_sms,
                                               small_queries=small_queries, pin=pin, mem_budget=mem_budget)
    res = {}
    for i, r in enumerate(reqs):
        q0, q1 = int(req_q[i]), int(req_q[i + 1])
        rr = Result(r.rid, r.arrival, float(launched[i]), float(done[i]), status=int(status[i]),
                    device=float(device[i]))
        if rr.status == 0:
            rr.ids, rr.scores = ids[q0:q1], sc[q0:q1]
        res[r.rid] = rr
    # batches issued at distinct instants (batches formed in the same pass of the loop count once)
    n_batches = len({float(t) for t, st in zip(launched, status) if st == 0})
    return list(res.values()), summarize(reqs, res, n_batches)


def serve(requests: list[Request], executor, *, topk: int, slots: int = 4, mem_budget: int = 16 << 30,
          max_batch_queries: int = 1 << 16, realtime: bool = True) -> tuple[list[Result], dict]:
    """Run the request stream through the executor; returns per-request results and a summary."""
    bat = Batcher(slots, topk, mem_budget, max_batch_queries)
    res = {r.rid: Result(r.rid, r.arrival) for r in requests}
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    t0 = time.perf_counter()
    n_batches = 0
    t_launch = t_collect = 0.0  # host seconds spent launching and collecting batches
    while pending or bat.busy():
        now = time.perf_counter() - t0 if realtime else math.inf
        while pending and pending[0].arrival <= now:
            bat.arrive(pending.popleft())
        for s, b in enumerate(bat.inflight):
            if b is not None and executor.done(b.handle):
                tc = time.perf_counter()
                ids, sc, t_done = executor.collect(b.handle)
                span = executor.device_span(b.handle) if hasattr(executor, "device_span") else math.nan
                bat.finish(s)
                q = 0
                for r in b.reqs:
                    rr = res[r.rid]
                    rr.ids, rr.scores = ids[q:q + r.nq], sc[q:q + r.nq]
                    rr.launched, rr.done, rr.device = b.launched, t_done - t0, span
                    q += r.nq
                t_collect += time.perf_counter() - tc
        if realtime:
            for r in bat.expire(time.perf_counter() - t0):
                res[r.rid].status = SLASH_ETIMEOUT
        for s in bat.free_slots():
            b = bat.next_batch(s)
            if b is None:
                break
            tl = time.perf_counter()
            b.launched = tl - t0
            if hasattr(executor, "launch_reqs"):
                b.handle = executor.launch_reqs(s, b.reqs)
            else:
                offs, cols = concat_csr(b.reqs)
                b.handle = executor.launch(s, offs, cols)
            t_launch += time.perf_counter() - tl
            n_batches += 1
        if not bat.queue and pending and realtime:
            wait = pending[0].arrival - (time.perf_counter() - t0)
            if wait > 2e-4 and not any(b is not None for b in bat.inflight):
                time.sleep(wait - 1e-4)
    for r in bat.refused:
        res[r.rid].status = SLASH_EBUSY
    summary = summarize(requests, res, n_batches)
    # host cost per batch of the loop's two calls into the executor
    summary["host_launch_us_per_batch"] = 1e6 * t_launch / max(1, n_batches)
    summary["host_collect_us_per_batch"] = 1e6 * t_collect / max(1, n_batches)
    return list(res.values()), summary


def poisson_requests(rate: float, n: int, pool_offs: np.ndarray, pool_cols: np.ndarray, *, seed: int = 0,
                     max_size: int = 4096, start: float = 0.0, timeout: float = math.inf) -> list[Request]:
    """n requests with exponential inter-arrival times (rate per second) and
    log-uniform sizes floor(max_size^u) in [1, max_size], cut from a query pool;
    each must be launched within `timeout` seconds of its arrival."""
    rng = np.random.default_rng(seed)
    t = start + np.cumsum(rng.exponential(1.0 / rate, n))
    sizes = np.clip(np.floor(max_size ** rng.random(n)).astype(np.int64), 1, max_size)
    npool = len(pool_offs) - 1
    out = []
    for i in range(n):
        a = int(rng.integers(0, max(1, npool - sizes[i])))
        b = min(npool, a + int(sizes[i]))
        o = pool_offs[a:b + 1]
        c = pool_cols[int(o[0]):int(o[-1])]
        out.append(Request(i, (o - o[0]).astype(np.uint64), c, float(t[i]), float(t[i]) + timeout))
    return out

"""Serving loop: continuous batching of query requests against a resident index.

Requests (each a CSR batch of 1..4096 queries) arrive over time.  The loop
keeps the index resident on the device and runs up to ``slots`` batches at
once, each on its own CUDA stream, so batches overlap on the device.  Whenever
a slot finishes, the requests that arrived meanwhile are admitted in arrival
order into the next batch, as long as the batch stays under
``max_batch_queries`` and the device bytes of all in-flight batches (CSR
inputs + outputs) stay under ``mem_budget``.  A request that could never fit
is refused (``SLASH_EBUSY``).  Latency = completion on the device - arrival.

The batching logic (:class:`Batcher`) is host code with no device calls; the
device work is behind :class:`GpuExecutor`, which issues the fused query
kernel through the C ABI.  Results do not depend on how requests are grouped:
every query is answered by one CTA from the same read-only index.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

SLASH_EBUSY = -5


@dataclass
class Request:
    rid: int
    offs: np.ndarray          # uint64 [nq+1], offs[0] == 0
    cols: np.ndarray          # uint32 [nnz]
    arrival: float            # seconds since the start of the run

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


def concat_csr(reqs: list[Request]) -> tuple[np.ndarray, np.ndarray]:
    nqs = [r.nq for r in reqs]
    offs = np.zeros(sum(nqs) + 1, dtype=np.uint64)
    pos, base = 0, 0
    for r in reqs:
        offs[pos + 1:pos + r.nq + 1] = r.offs[1:] + base
        pos += r.nq
        base += len(r.cols)
    cols = np.concatenate([r.cols for r in reqs]) if reqs else np.zeros(0, np.uint32)
    return offs, cols


class GpuExecutor:
    """One CUDA stream per slot; H2D of the batch, fused query, D2H of the results."""

    def __init__(self, ix, topk: int, slots: int, threads: int = 0):
        import torch
        self.torch = torch
        self.ix, self.topk, self.threads = ix, topk, threads
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.ref = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        self.ref.record(torch.cuda.current_stream())
        self.ref.synchronize()
        self.t_ref = time.perf_counter()

    def launch(self, slot: int, offs: np.ndarray, cols: np.ndarray):
        torch = self.torch
        st = self.streams[slot]
        nq = len(offs) - 1
        with torch.cuda.stream(st):
            h_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
            h_cols = torch.from_numpy(cols.view(np.int32)).pin_memory()
            d_offs = h_offs.to("cuda", non_blocking=True)
            d_cols = h_cols.to("cuda", non_blocking=True)
            d_ids = torch.empty((nq, self.topk), dtype=torch.int32, device="cuda")
            d_sc = torch.empty_like(d_ids)
            self.ix.query(d_offs, d_cols, self.topk, st, d_ids_out=d_ids, d_scores_out=d_sc, mode="fused",
                          threads=self.threads)
            h_ids = torch.empty((nq, self.topk), dtype=torch.int32, pin_memory=True)
            h_sc = torch.empty((nq, self.topk), dtype=torch.int32, pin_memory=True)
            h_ids.copy_(d_ids, non_blocking=True)
            h_sc.copy_(d_sc, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
        # keep every buffer alive until the event completes
        return (ev, h_offs, h_cols, d_offs, d_cols, d_ids, d_sc, h_ids, h_sc)

    def done(self, h) -> bool:
        return h[0].query()

    def collect(self, h) -> tuple[np.ndarray, np.ndarray, float]:
        ev = h[0]
        ev.synchronize()
        t_done = self.t_ref + self.ref.elapsed_time(ev) / 1e3
        return h[7].numpy(), h[8].numpy().view(np.uint32), t_done


def serve(requests: list[Request], executor, *, topk: int, slots: int = 4, mem_budget: int = 16 << 30,
          max_batch_queries: int = 1 << 16, realtime: bool = True) -> tuple[list[Result], dict]:
    """Run the request stream through the executor; returns per-request results and a summary."""
    bat = Batcher(slots, topk, mem_budget, max_batch_queries)
    res = {r.rid: Result(r.rid, r.arrival) for r in requests}
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    t0 = time.perf_counter()
    n_batches = 0
    while pending or bat.busy():
        now = time.perf_counter() - t0 if realtime else math.inf
        while pending and pending[0].arrival <= now:
            bat.arrive(pending.popleft())
        for s, b in enumerate(bat.inflight):
            if b is not None and executor.done(b.handle):
                ids, sc, t_done = executor.collect(b.handle)
                bat.finish(s)
                q = 0
                for r in b.reqs:
                    rr = res[r.rid]
                    rr.ids, rr.scores = ids[q:q + r.nq], sc[q:q + r.nq]
                    rr.launched, rr.done = b.launched, t_done - t0
                    q += r.nq
        for s in bat.free_slots():
            b = bat.next_batch(s)
            if b is None:
                break
            offs, cols = concat_csr(b.reqs)
            b.launched = time.perf_counter() - t0
            b.handle = executor.launch(s, offs, cols)
            n_batches += 1
        if not bat.queue and pending and realtime:
            wait = pending[0].arrival - (time.perf_counter() - t0)
            if wait > 2e-4 and not any(b is not None for b in bat.inflight):
                time.sleep(wait - 1e-4)
    for r in bat.refused:
        res[r.rid].status = SLASH_EBUSY
    done = [r for r in res.values() if r.status == 0]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    nq = sum(q.nq for q in requests if res[q.rid].status == 0)
    span = max(r.done for r in done) - min(r.arrival for r in done) if done else 1.0
    summary = {"requests": len(done), "refused": len(bat.refused), "queries": nq, "batches": n_batches,
               "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
               "mean_ms": 1e3 * float(lat.mean()), "queries_per_s": nq / span if span > 0 else float("nan"),
               "span_s": span}
    return list(res.values()), summary


def poisson_requests(rate: float, n: int, pool_offs: np.ndarray, pool_cols: np.ndarray, *, seed: int = 0,
                     max_size: int = 4096, start: float = 0.0) -> list[Request]:
    """n requests with exponential inter-arrival times (rate per second) and
    log-uniform sizes floor(max_size^u) in [1, max_size], cut from a query pool."""
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
        out.append(Request(i, (o - o[0]).astype(np.uint64), c, float(t[i])))
    return out

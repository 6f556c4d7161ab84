"""Python binding of ``libslash.so`` -- the SLASH hot path on one B300.

Argument marshalling only: every step of hashing, insertion and querying runs
in the library's CUDA kernels (see ``include/slash.h``).  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is
missing or fails to load, importing this package raises.

The functions carry the C ABI's names::

    ix = slash_build_index(params)                       # -> handle
    first = slash_insert(ix, d_offs, d_cols)             # Algorithm 1
    ids, scores = slash_query(ix, d_offs, d_cols, topk)  # Algorithm 2
    slash_free(ix)

``d_offs`` is an 8-byte integer CUDA tensor of n+1 CSR offsets, ``d_cols`` a
4-byte integer CUDA tensor of feature ids; both are passed by pointer.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# SLASH_CHECKED=1 loads the checked build (bounds-tested indices; slower)
_CHECKED = os.environ.get("SLASH_CHECKED", "") == "1"
_LIB_PATH = os.path.join(_PKG, "libslash_checked.so" if _CHECKED else "libslash.so")

SLASH_OK = 0
SLASH_EINVAL = -1
SLASH_ENOMEM = -2
SLASH_ECUDA = -3
SLASH_EFULL = -4
SLASH_EBUSY = -5
SLASH_ETIMEOUT = -6
SLASH_EDATA = -7
SLASH_EIO = -8
SLASH_DENSIFY_SIDE = 0
SLASH_DENSIFY_OPTIMAL = 1
SLASH_EMPTY = 0xFFFFFFFF
SLASH_MAX_TOPK = 256


class SlashError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {slash_strerror(code)} ({code})")


SLASH_SERVE_NO_PIN = 1  # slash_serve_opts.flags (include/slash_serve.h)
SLASH_QUERY_FUSED = 0
SLASH_QUERY_PLAIN = 1
SLASH_QUERY_WARP_FUSED = 2
SLASH_QUERY_WARP_PLAIN = 3
_MODES = {"fused": SLASH_QUERY_FUSED, "plain": SLASH_QUERY_PLAIN, "warp_fused": SLASH_QUERY_WARP_FUSED,
          "warp_plain": SLASH_QUERY_WARP_PLAIN}


class slash_query_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("max_sms", ctypes.c_uint32)]

    def __repr__(self):
        m = {v: k for k, v in _MODES.items()}.get(self.mode, str(self.mode))
        return (f"slash_query_opts({m}, threads={self.threads}, ctas_per_sm={self.ctas_per_sm}, "
                f"max_sms={self.max_sms})")


# the allocator hook's callback types (include/slash.h)
SLASH_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
SLASH_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class slash_serve_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("max_batch_queries", ctypes.c_uint32), ("topk", ctypes.c_uint32),
                ("mode", ctypes.c_uint32), ("threads", ctypes.c_uint32), ("reserve_sms", ctypes.c_uint32),
                ("small_queries", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("timeout_s", ctypes.c_double),
                ("mem_budget_bytes", ctypes.c_uint64)]


class slash_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_uint32), ("K", ctypes.c_uint32), ("L", ctypes.c_uint32),
                ("log2_buckets", ctypes.c_uint32), ("reservoir", ctypes.c_uint32),
                ("cm_rows", ctypes.c_uint32), ("cm_width", ctypes.c_uint32),
                ("shards", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("capacity", ctypes.c_uint64), ("densify", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class slash_tk_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_uint32), ("K", ctypes.c_uint32), ("L", ctypes.c_uint32),
                ("log2_buckets", ctypes.c_uint32), ("rows", ctypes.c_uint32), ("cells", ctypes.c_uint32),
                ("shards", ctypes.c_uint32), ("densify", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("capacity", ctypes.c_uint64)]


def _load() -> ctypes.CDLL:
    from . import build as _build
    if _build.needs_build(_CHECKED):  # compile the CUDA library in place (nvcc); no fallback if that fails
        _build.build(checked=_CHECKED)
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libslash.so not built ({_LIB_PATH}); run python -m paper_2008_03260_b300.build")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "slash_build_index": (i32, [P(slash_params), vp, P(vp)]),
        "slash_insert": (i32, [vp, vp, vp, u32, P(u64), vp]),
        "slash_query": (i32, [vp, vp, vp, u32, u32, vp, vp, vp]),
        "slash_insert_host": (i32, [vp, vp, vp, u32, P(u64), vp]),
        "slash_free": (i32, [vp]),
        "slash_strerror": (ctypes.c_char_p, [i32]),
        "slash_sync": (i32, [vp, vp]),
        "slash_reset": (i32, [vp, vp]),
        "slash_size": (u64, [vp]),
        "slash_debug_hash": (i32, [vp, vp, vp, u32, vp, vp, vp]),
        "slash_debug_export": (i32, [vp, vp, vp]),
        "slash_debug_fail_alloc": (i32, [vp, u32]),
        "slash_debug_occupancy": (i32, [vp, u32, u32, P(ctypes.c_int)]),
        "slash_probe_smem": (i32, [u32, u32, u32, u32, u32, P(ctypes.c_float), P(u64)]),
        "slash_set_next_id": (i32, [vp, u64]),
        "slash_query_candidates": (i32, [vp, vp, vp, u32, u32, vp, vp, vp]),
        "slash_query_cells": (i32, [vp, vp, vp, u32, u32, u32, vp, vp, vp, vp]),
        "slash_rank_candidates": (i32, [u32, u32, u32, u32, vp, vp, vp, u32, vp, vp, vp]),
        "slash_debug_stall_copies": (i32, [vp, i32]),
        "slash_debug_buckets": (i32, [vp, vp, vp, vp, u32, vp, vp]),
        "slash_query_ex": (i32, [vp, vp, vp, u32, u32, vp, vp, P(slash_query_opts), vp]),
        "slash_autotune": (i32, [vp, vp, vp, u32, u32, vp, vp, vp, P(slash_query_opts), P(ctypes.c_float)]),
        "slash_query_static": (i32, [vp, vp, vp, u32, u32, vp, vp, vp]),
        "slash_serve": (i32, [vp, P(slash_serve_opts), u32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "slash_set_allocator": (i32, [vp, SLASH_ALLOC_FN, SLASH_FREE_FN, vp]),
        "slash_debug_bounds": (i32, [P(u32), P(u32)]),
        "slash_profile": (i32, [vp, i32]),
        "slash_profile_read": (i32, [vp, u32, vp, vp, vp, P(u32), P(u64)]),
        "slash_tk_build": (i32, [P(slash_tk_params), vp, P(vp)]),
        "slash_tk_insert": (i32, [vp, vp, vp, u32, P(u64), vp]),
        "slash_tk_query": (i32, [vp, vp, vp, u32, u32, u32, vp, vp, vp]),
        "slash_tk_export": (i32, [vp, vp]),
        "slash_tk_sync": (i32, [vp, vp]),
        "slash_tk_reset": (i32, [vp, vp]),
        "slash_tk_size": (u64, [vp]),
        "slash_tk_launches": (u64, [vp]),
        "slash_tk_free": (i32, [vp]),
        "slash_tk_debug_buckets": (i32, [vp, vp, vp, vp, u32, vp]),
        "slash_save": (i32, [vp, ctypes.c_char_p]),
        "slash_load": (i32, [ctypes.c_char_p, vp, P(vp)]),
        "slash_get_params": (i32, [vp, P(slash_params)]),
        "slash_tk_save": (i32, [vp, ctypes.c_char_p]),
        "slash_tk_load": (i32, [ctypes.c_char_p, vp, P(vp)]),
        "slash_tk_get_params": (i32, [vp, P(slash_tk_params)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


_lib = _load()


def library_path() -> str:
    return _LIB_PATH


def _check(rc: int, where: str) -> None:
    if rc != SLASH_OK:
        raise SlashError(rc, where)


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream or None
    return int(stream) or None


def _dev_ptr(t: torch.Tensor, itemsize: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.element_size() != itemsize or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous with {itemsize}-byte elements")
    return t.data_ptr()


@dataclass(frozen=True)
class Params:
    """Index parameters (see ``slash_params`` in include/slash.h)."""
    dim: int = 1 << 20
    K: int = 4
    L: int = 16
    log2_buckets: int = 16
    reservoir: int = 32
    cm_rows: int = 4
    cm_width: int = 4096
    shards: int = 1
    seed: int = 0
    capacity: int = 100_000
    densify: int = 0  # SLASH_DENSIFY_SIDE (0) or SLASH_DENSIFY_OPTIMAL (1)

    def c(self) -> slash_params:
        return slash_params(self.dim, self.K, self.L, self.log2_buckets, self.reservoir,
                            self.cm_rows, self.cm_width, self.shards, self.seed, self.capacity,
                            self.densify, 0)

    @property
    def index_bytes(self) -> int:
        nk = self.shards * self.L << self.log2_buckets
        return nk * (self.reservoir + 1) * 4


# --------------------------------------------------------------------------- C-ABI names
def slash_strerror(code: int) -> str:
    return _lib.slash_strerror(code).decode()


def slash_build_index(p: Params, stream=None) -> int:
    h = ctypes.c_void_p()
    cp = p.c()
    _check(_lib.slash_build_index(ctypes.byref(cp), _stream(stream), ctypes.byref(h)),
           "slash_build_index")
    return h.value


def slash_insert(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, stream=None) -> int:
    n = d_offs.numel() - 1
    if n < 0:
        raise ValueError("d_offs needs n+1 entries")
    first = ctypes.c_uint64()
    _check(_lib.slash_insert(ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), n,
                             ctypes.byref(first), _stream(stream)), "slash_insert")
    return int(first.value)


def slash_insert_host(ix: int, h_offs: torch.Tensor, h_cols: torch.Tensor, stream=None) -> int:
    """Insert rows held in (preferably pinned) host memory; copies overlap the hashing."""
    if h_offs.is_cuda or h_cols.is_cuda:
        raise TypeError("slash_insert_host takes host tensors")
    if h_offs.element_size() != 8 or h_cols.element_size() != 4 or not (h_offs.is_contiguous() and
                                                                        h_cols.is_contiguous()):
        raise TypeError("h_offs: contiguous 8-byte ints, h_cols: contiguous 4-byte ints")
    n = h_offs.numel() - 1
    first = ctypes.c_uint64()
    _check(_lib.slash_insert_host(ix, h_offs.data_ptr(), h_cols.data_ptr(), n, ctypes.byref(first),
                                  _stream(stream)), "slash_insert_host")
    return int(first.value)


def _opts(mode, threads, ctas_per_sm, max_sms=0):
    if mode is None:
        return None
    m = _MODES.get(mode, mode)
    return slash_query_opts(int(m), int(threads or 0), int(ctas_per_sm or 0), int(max_sms or 0))


def slash_query(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, topk: int,
                d_ids_out: torch.Tensor | None = None, d_scores_out: torch.Tensor | None = None,
                stream=None, mode=None, threads: int = 0, ctas_per_sm: int = 0, max_sms: int = 0
                ) -> tuple[torch.Tensor, torch.Tensor]:
    """Algorithm 2 for a batch.  ``mode`` None = the index's default schedule,
    else "fused" / "plain" / "warp_fused" / "warp_plain" (with optional
    ``threads``, ``ctas_per_sm`` and ``max_sms``)."""
    nq = d_offs.numel() - 1
    if nq < 0:
        raise ValueError("d_offs needs n+1 entries")
    dev = d_offs.device
    if d_ids_out is None:
        d_ids_out = torch.empty((nq, topk), dtype=torch.int32, device=dev)
    if d_scores_out is None:
        d_scores_out = torch.empty((nq, topk), dtype=torch.int32, device=dev)
    if d_ids_out.numel() < nq * topk or d_scores_out.numel() < nq * topk:
        raise ValueError("output tensors too small")
    o = _opts(mode, threads, ctas_per_sm, max_sms)
    args = (ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), nq, topk,
            _dev_ptr(d_ids_out, 4, "d_ids_out"), _dev_ptr(d_scores_out, 4, "d_scores_out"))
    if o is None:
        _check(_lib.slash_query(*args, _stream(stream)), "slash_query")
    else:
        _check(_lib.slash_query_ex(*args, ctypes.byref(o), _stream(stream)), "slash_query_ex")
    return d_ids_out, d_scores_out


def slash_autotune(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, topk: int, stream=None):
    """Time every query schedule on this sample batch; the fastest becomes the
    index default.  Returns (opts, best ms)."""
    nq = d_offs.numel() - 1
    ids = torch.empty((nq, topk), dtype=torch.int32, device=d_offs.device)
    sc = torch.empty_like(ids)
    best = slash_query_opts()
    ms = ctypes.c_float()
    _check(_lib.slash_autotune(ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), nq, topk,
                               ids.data_ptr(), sc.data_ptr(), _stream(stream), ctypes.byref(best),
                               ctypes.byref(ms)), "slash_autotune")
    return best, float(ms.value)


def slash_serve(ix: int, arrival_s, req_q, offs, cols, topk: int, *, slots: int = 4,
                max_batch_queries: int = 8192, mode="fused", threads: int = 0, timeout_s: float = 0.0,
                reserve_sms: int = 0, small_queries: int = 0, pin: bool = True, mem_budget: int = 0):
    """The native serving loop (include/slash_serve.h) over host arrays:
    arrival_s float64 [n], req_q uint64 [n+1] (request i = queries
    [req_q[i], req_q[i+1])), the queries' CSR offs uint64 / cols uint32.
    Returns (ids int32 [Q][topk], scores uint32 [Q][topk], launched_s, done_s,
    status int32, device_s), one time, status and batch device span per request."""
    import numpy as np
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    rq = np.ascontiguousarray(req_q, dtype=np.uint64)
    of = np.ascontiguousarray(offs, dtype=np.uint64)
    co = np.ascontiguousarray(cols, dtype=np.uint32)
    n = arr.size
    if rq.size != n + 1:
        raise ValueError("req_q needs n_requests + 1 entries")
    nq = int(rq[-1]) if n else 0
    ids = np.empty((nq, topk), dtype=np.int32)
    sc = np.empty((nq, topk), dtype=np.uint32)
    launched = np.empty(n, dtype=np.float64)
    done = np.empty(n, dtype=np.float64)
    status = np.empty(n, dtype=np.int32)
    device = np.empty(n, dtype=np.float64)
    o = slash_serve_opts(slots, max_batch_queries, topk, _MODES.get(mode, mode), threads, reserve_sms,
                         small_queries, 0 if pin else SLASH_SERVE_NO_PIN, timeout_s, mem_budget)
    ptr = lambda a: a.ctypes.data if a.size else None
    _check(_lib.slash_serve(ix, ctypes.byref(o), n, ptr(arr), rq.ctypes.data, of.ctypes.data, ptr(co), ptr(ids),
                            ptr(sc), ptr(launched), ptr(done), ptr(status), ptr(device)), "slash_serve")
    return ids, sc, launched, done, status, device


def slash_set_allocator(ix: int, alloc=None, release=None) -> None:
    """Route the index's workspace through alloc(bytes) -> device pointer (0 or
    None when out of memory) and release(ptr); both None restores cudaMalloc.
    Keep the returned callback objects alive as long as the index uses them."""
    if (alloc is None) != (release is None):
        raise ValueError("give both alloc and release, or neither")
    if alloc is None:
        _check(_lib.slash_set_allocator(ix, SLASH_ALLOC_FN(), SLASH_FREE_FN(), None), "slash_set_allocator")
        return None

    def _a(n, ctx):
        try:
            return alloc(int(n)) or None
        except Exception:  # an exception cannot cross the C boundary: report no memory
            return None

    def _f(ptr, ctx):
        release(int(ptr))

    cbs = (SLASH_ALLOC_FN(_a), SLASH_FREE_FN(_f))
    _check(_lib.slash_set_allocator(ix, cbs[0], cbs[1], None), "slash_set_allocator")
    return cbs


def slash_debug_bounds() -> tuple[bool, int]:
    """(is this the checked build, its out-of-range flag since the last call); clears the flag."""
    c, e = ctypes.c_uint32(), ctypes.c_uint32()
    _check(_lib.slash_debug_bounds(ctypes.byref(c), ctypes.byref(e)), "slash_debug_bounds")
    return bool(c.value), int(e.value)


def torch_allocator():
    """(alloc, release) over PyTorch's caching allocator on the current device
    and stream, for slash_set_allocator / Index.set_allocator."""
    import torch
    return (lambda n: torch.cuda.caching_allocator_alloc(n), lambda p: torch.cuda.caching_allocator_delete(p))


def slash_free(ix: int) -> None:
    if ix:
        _check(_lib.slash_free(ix), "slash_free")


def slash_sync(ix: int, stream=None) -> int:
    return int(_lib.slash_sync(ix, _stream(stream)))


def slash_reset(ix: int, stream=None) -> None:
    _check(_lib.slash_reset(ix, _stream(stream)), "slash_reset")


def slash_size(ix: int) -> int:
    return int(_lib.slash_size(ix))


def slash_debug_hash(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, nb: int, L: int,
                     want_codes: bool = True, stream=None):
    n = d_offs.numel() - 1
    dev = d_offs.device
    codes = torch.empty((n, nb), dtype=torch.int32, device=dev) if want_codes else None
    bk = torch.empty((L, n), dtype=torch.int32, device=dev)
    _check(_lib.slash_debug_hash(ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), n,
                                 codes.data_ptr() if codes is not None else None, bk.data_ptr(),
                                 _stream(stream)), "slash_debug_hash")
    return codes, bk


def slash_debug_fail_alloc(ix: int, count: int) -> None:
    """Test support: the index's next ``count`` workspace allocations fail (SLASH_ENOMEM)."""
    _check(_lib.slash_debug_fail_alloc(ix, count), "slash_debug_fail_alloc")


def slash_set_next_id(ix: int, next_id: int) -> None:
    """Rows inserted next take ids from next_id on (a partition starting at its global id)."""
    _check(_lib.slash_set_next_id(ix, next_id), "slash_set_next_id")


def slash_query_candidates(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, m: int, stream=None):
    """Each query's distinct local candidates: counts int32 [nq], ids int32 [nq, m] in the order of their
    first occurrence in the query's buckets, -1 past the count."""
    nq = d_offs.numel() - 1
    counts = torch.empty(nq, dtype=torch.int32, device=d_offs.device)
    ids = torch.empty((nq, m), dtype=torch.int32, device=d_offs.device)
    _check(_lib.slash_query_candidates(ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), nq, m,
                                       counts.data_ptr(), ids.data_ptr(), _stream(stream)), "slash_query_candidates")
    return counts, ids


def slash_query_cells(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, ids: torch.Tensor, counts: torch.Tensor,
                      d: int, stream=None) -> torch.Tensor:
    """This index's count-min cells of gathered candidates ids [W, nq, m] (counts [W, nq]): int32 [W, nq, m, d]."""
    W, nq, m = ids.shape
    cells = torch.empty((W, nq, m, d), dtype=torch.int32, device=ids.device)
    _check(_lib.slash_query_cells(ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), nq, W, m,
                                  _dev_ptr(counts, 4, "counts"), _dev_ptr(ids, 4, "ids"), cells.data_ptr(),
                                  _stream(stream)), "slash_query_cells")
    return cells


def slash_rank_candidates(ids: torch.Tensor, counts: torch.Tensor, cells: torch.Tensor, topk: int, stream=None):
    """Top-k (ids int32 [nq, k], scores int32 [nq, k]) from gathered ids and their summed cells."""
    W, nq, m = ids.shape
    d = cells.shape[-1]
    out_ids = torch.empty((nq, topk), dtype=torch.int32, device=ids.device)
    out_sc = torch.empty((nq, topk), dtype=torch.int32, device=ids.device)
    _check(_lib.slash_rank_candidates(W, nq, m, d, _dev_ptr(counts, 4, "counts"), _dev_ptr(ids, 4, "ids"),
                                      _dev_ptr(cells, 4, "cells"), topk, out_ids.data_ptr(), out_sc.data_ptr(),
                                      _stream(stream)), "slash_rank_candidates")
    return out_ids, out_sc


def slash_probe_smem(mode: int, words: int = 16384, iters: int = 4096, threads: int = 512,
                     ctas_per_sm: int = 2) -> tuple[float, int]:
    """Shared-memory microbenchmark (see include/slash.h): (ms, operations)."""
    ms, ops = ctypes.c_float(), ctypes.c_uint64()
    _check(_lib.slash_probe_smem(mode, words, iters, threads, ctas_per_sm, ctypes.byref(ms), ctypes.byref(ops)),
           "slash_probe_smem")
    return float(ms.value), int(ops.value)


def slash_debug_occupancy(ix: int, mode, threads: int) -> int:
    """Test support: CTAs per SM the occupancy calculator allows the query kernel of a schedule."""
    m = _MODES.get(mode, mode)
    out = ctypes.c_int()
    _check(_lib.slash_debug_occupancy(ix, int(m), threads, ctypes.byref(out)), "slash_debug_occupancy")
    return int(out.value)


def slash_debug_stall_copies(ix: int, enable: bool) -> None:
    """Test support: staged query waits give up after their time limit (SLASH_ETIMEOUT)."""
    _check(_lib.slash_debug_stall_copies(ix, 1 if enable else 0), "slash_debug_stall_copies")


def slash_debug_export(ix: int, p: Params, fill_only: bool = False):
    import numpy as np
    nk = p.shards * p.L << p.log2_buckets
    slots = None if fill_only else np.empty(nk * p.reservoir, dtype=np.uint32)
    fill = np.empty(nk, dtype=np.uint32)
    _check(_lib.slash_debug_export(ix, None if slots is None else slots.ctypes.data, fill.ctypes.data),
           "slash_debug_export")
    return (None if slots is None else slots.reshape(p.shards, p.L, 1 << p.log2_buckets, p.reservoir),
            fill.reshape(p.shards, p.L, 1 << p.log2_buckets))


def slash_debug_buckets(ix: int, p: Params, shard, table, bucket):
    import numpy as np
    s = np.ascontiguousarray(shard, dtype=np.uint32)
    t = np.ascontiguousarray(table, dtype=np.uint32)
    b = np.ascontiguousarray(bucket, dtype=np.uint32)
    n = s.size
    slots = np.empty((n, p.reservoir), dtype=np.uint32)
    fill = np.empty(n, dtype=np.uint32)
    _check(_lib.slash_debug_buckets(ix, s.ctypes.data, t.ctypes.data, b.ctypes.data, n,
                                    slots.ctypes.data, fill.ctypes.data), "slash_debug_buckets")
    return slots, fill


def slash_profile(ix: int, enable: bool) -> None:
    _check(_lib.slash_profile(ix, 1 if enable else 0), "slash_profile")


def slash_profile_read(ix: int, max_kernels: int = 32) -> tuple[dict, int]:
    """{kernel name: (total ms, launches)} since profiling was enabled, and the
    index's total kernel launches since it was built."""
    names = ctypes.create_string_buffer(32 * max_kernels)
    ms = (ctypes.c_float * max_kernels)()
    cnt = (ctypes.c_uint32 * max_kernels)()
    n = ctypes.c_uint32()
    tot = ctypes.c_uint64()
    _check(_lib.slash_profile_read(ix, max_kernels, names, ms, cnt, ctypes.byref(n), ctypes.byref(tot)),
           "slash_profile_read")
    out = {}
    for i in range(min(n.value, max_kernels)):
        nm = names.raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(cnt[i]))
    return out, int(tot.value)


def slash_save(ix: int, path: str) -> None:
    _check(_lib.slash_save(ix, os.fsencode(path)), "slash_save")


def slash_load(path: str, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(_lib.slash_load(os.fsencode(path), _stream(stream), ctypes.byref(h)), "slash_load")
    return h.value


def slash_get_params(ix: int) -> Params:
    cp = slash_params()
    _check(_lib.slash_get_params(ix, ctypes.byref(cp)), "slash_get_params")
    return Params(**{f: getattr(cp, f) for f, _ in slash_params._fields_ if f != "reserved"})


class Index:
    """Owning wrapper: ``Index(Params(...))``, ``.insert``, ``.query``, ``.close``;
    ``Index.load(path)`` reopens a ``.save(path)`` checkpoint."""

    def __init__(self, p: Params | None, stream=None, _handle: int | None = None):
        if _handle is not None:
            self.h = _handle
            self.p = slash_get_params(_handle)
        else:
            self.p = p
            self.h = slash_build_index(p, stream)

    @classmethod
    def load(cls, path: str, stream=None) -> "Index":
        return cls(None, stream, _handle=slash_load(path, stream))

    def save(self, path: str) -> None:
        slash_save(self.h, path)

    def insert(self, d_offs, d_cols, stream=None) -> int:
        return slash_insert(self.h, d_offs, d_cols, stream)

    def set_next_id(self, next_id: int) -> None:
        slash_set_next_id(self.h, next_id)

    def insert_host(self, h_offs, h_cols, stream=None) -> int:
        return slash_insert_host(self.h, h_offs, h_cols, stream)

    def query(self, d_offs, d_cols, topk: int, stream=None, **kw):
        return slash_query(self.h, d_offs, d_cols, topk, stream=stream, **kw)

    def autotune(self, d_offs, d_cols, topk: int, stream=None):
        return slash_autotune(self.h, d_offs, d_cols, topk, stream)

    def serve(self, arrival_s, req_q, offs, cols, topk: int, **kw):
        return slash_serve(self.h, arrival_s, req_q, offs, cols, topk, **kw)

    def sync(self, stream=None) -> None:
        _check(slash_sync(self.h, stream), "slash_sync")

    def reset(self, stream=None) -> None:
        slash_reset(self.h, stream)

    @property
    def size(self) -> int:
        return slash_size(self.h)

    def export(self, fill_only: bool = False):
        return slash_debug_export(self.h, self.p, fill_only)

    def buckets(self, shard, table, bucket):
        return slash_debug_buckets(self.h, self.p, shard, table, bucket)

    def debug_hash(self, d_offs, d_cols, want_codes: bool = True, stream=None):
        return slash_debug_hash(self.h, d_offs, d_cols, self.p.K * self.p.L, self.p.L, want_codes, stream)

    def profile(self, enable: bool = True) -> None:
        slash_profile(self.h, enable)

    def profile_read(self) -> tuple[dict, int]:
        return slash_profile_read(self.h)

    def set_allocator(self, alloc=None, release=None) -> None:
        """The index's workspace from alloc / release (see slash_set_allocator);
        Index.set_allocator(*torch_allocator()) uses PyTorch's caching allocator."""
        self._alloc_cbs = slash_set_allocator(self.h, alloc, release)

    def close(self) -> None:
        h, self.h = self.h, None
        if h:
            slash_free(h)
        self._alloc_cbs = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- TopKAPI buckets
@dataclass(frozen=True)
class TkParams:
    """Sketch-bucket index parameters (see ``slash_tk_params`` in include/slash_topkapi.h)."""
    dim: int = 1 << 20
    K: int = 4
    L: int = 16
    log2_buckets: int = 12
    rows: int = 4
    cells: int = 32
    shards: int = 1
    seed: int = 0
    capacity: int = 100_000
    densify: int = 0  # SLASH_DENSIFY_SIDE (0) or SLASH_DENSIFY_OPTIMAL (1)

    def c(self) -> slash_tk_params:
        return slash_tk_params(self.dim, self.K, self.L, self.log2_buckets, self.rows, self.cells,
                               self.shards, self.densify, self.seed, self.capacity)

    @property
    def index_bytes(self) -> int:
        return (self.shards * self.L << self.log2_buckets) * self.rows * self.cells * 4


def slash_tk_build(p: TkParams, stream=None) -> int:
    h = ctypes.c_void_p()
    cp = p.c()
    _check(_lib.slash_tk_build(ctypes.byref(cp), _stream(stream), ctypes.byref(h)), "slash_tk_build")
    return h.value


def slash_tk_insert(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, stream=None) -> int:
    n = d_offs.numel() - 1
    if n < 0:
        raise ValueError("d_offs needs n+1 entries")
    first = ctypes.c_uint64()
    _check(_lib.slash_tk_insert(ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), n,
                                ctypes.byref(first), _stream(stream)), "slash_tk_insert")
    return int(first.value)


def slash_tk_query(ix: int, d_offs: torch.Tensor, d_cols: torch.Tensor, topk: int, threshold: int = 0,
                   d_ids_out: torch.Tensor | None = None, d_scores_out: torch.Tensor | None = None,
                   stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    nq = d_offs.numel() - 1
    if nq < 0:
        raise ValueError("d_offs needs n+1 entries")
    dev = d_offs.device
    if d_ids_out is None:
        d_ids_out = torch.empty((nq, topk), dtype=torch.int32, device=dev)
    if d_scores_out is None:
        d_scores_out = torch.empty((nq, topk), dtype=torch.int32, device=dev)
    if d_ids_out.numel() < nq * topk or d_scores_out.numel() < nq * topk:
        raise ValueError("output tensors too small")
    _check(_lib.slash_tk_query(ix, _dev_ptr(d_offs, 8, "d_offs"), _dev_ptr(d_cols, 4, "d_cols"), nq, topk,
                               threshold, _dev_ptr(d_ids_out, 4, "d_ids_out"),
                               _dev_ptr(d_scores_out, 4, "d_scores_out"), _stream(stream)), "slash_tk_query")
    return d_ids_out, d_scores_out


def slash_tk_export(ix: int, p: TkParams):
    """Cell words [S][L][2^B][W][C]: 0 = empty, else heavy hitter id + 1 (count 1)."""
    import numpy as np
    out = np.empty((p.shards, p.L, 1 << p.log2_buckets, p.rows, p.cells), dtype=np.uint32)
    _check(_lib.slash_tk_export(ix, out.ctypes.data), "slash_tk_export")
    return out


def slash_tk_free(ix: int) -> None:
    if ix:
        _check(_lib.slash_tk_free(ix), "slash_tk_free")


def slash_tk_save(ix: int, path: str) -> None:
    _check(_lib.slash_tk_save(ix, os.fsencode(path)), "slash_tk_save")


def slash_tk_load(path: str, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(_lib.slash_tk_load(os.fsencode(path), _stream(stream), ctypes.byref(h)), "slash_tk_load")
    return h.value


def slash_tk_get_params(ix: int) -> TkParams:
    cp = slash_tk_params()
    _check(_lib.slash_tk_get_params(ix, ctypes.byref(cp)), "slash_tk_get_params")
    return TkParams(**{f: getattr(cp, f) for f, _ in slash_tk_params._fields_})


class TkIndex:
    """Owning wrapper of a sketch-bucket index: ``.insert``, ``.query``, ``.export``;
    ``TkIndex.load(path)`` reopens a ``.save(path)`` checkpoint."""

    def __init__(self, p: TkParams | None, stream=None, _handle: int | None = None):
        if _handle is not None:
            self.h = _handle
            self.p = slash_tk_get_params(_handle)
        else:
            self.p = p
            self.h = slash_tk_build(p, stream)

    @classmethod
    def load(cls, path: str, stream=None) -> "TkIndex":
        return cls(None, stream, _handle=slash_tk_load(path, stream))

    def save(self, path: str) -> None:
        slash_tk_save(self.h, path)

    def insert(self, d_offs, d_cols, stream=None) -> int:
        return slash_tk_insert(self.h, d_offs, d_cols, stream)

    def query(self, d_offs, d_cols, topk: int, threshold: int = 0, stream=None):
        return slash_tk_query(self.h, d_offs, d_cols, topk, threshold, stream=stream)

    def export(self):
        return slash_tk_export(self.h, self.p)

    def buckets(self, shard, table, bucket):
        """Cell words [n][W][C] of the listed sketches."""
        import numpy as np
        s_ = np.ascontiguousarray(shard, dtype=np.uint32)
        t_ = np.ascontiguousarray(table, dtype=np.uint32)
        b_ = np.ascontiguousarray(bucket, dtype=np.uint32)
        out = np.empty((s_.size, self.p.rows, self.p.cells), dtype=np.uint32)
        _check(_lib.slash_tk_debug_buckets(self.h, s_.ctypes.data, t_.ctypes.data, b_.ctypes.data, s_.size,
                                           out.ctypes.data), "slash_tk_debug_buckets")
        return out

    def sync(self, stream=None) -> None:
        _check(int(_lib.slash_tk_sync(self.h, _stream(stream))), "slash_tk_sync")

    def reset(self, stream=None) -> None:
        _check(_lib.slash_tk_reset(self.h, _stream(stream)), "slash_tk_reset")

    @property
    def size(self) -> int:
        return int(_lib.slash_tk_size(self.h))

    @property
    def launches(self) -> int:
        return int(_lib.slash_tk_launches(self.h))

    def close(self) -> None:
        h, self.h = self.h, None
        if h:
            slash_tk_free(h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

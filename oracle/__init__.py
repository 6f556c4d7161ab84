"""CPU oracle for the SLASH hot path (arXiv 2008.03260) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs anything here, and this
package imports nothing from the product path.

The arithmetic lives in ``slash_oracle.c`` (plain C, one obvious loop per step
of the paper's method, see its header for the fixed readings); this module is
ctypes marshalling plus numpy conveniences.

Parity pins (what ties the oracle to the paper rather than to itself) are in
``tests/test_oracle_pins.py``; every oracle function there has at least one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slash_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None
EMPTY = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (gcc -O2, no vendor code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
            lib.or_mix32.restype = u32
            lib.or_mix32.argtypes = [u32]
            lib.or_splitmix64_next.restype = u64
            lib.or_splitmix64_next.argtypes = [ctypes.POINTER(u64)]
            lib.or_derive_seeds.argtypes = [u64, u32, u32, vp]
            lib.or_minhash.restype = u32
            lib.or_minhash.argtypes = [vp, u64, u32]
            lib.or_doph.argtypes = [vp, u64, u32, u32, u32, vp, vp]
            lib.or_doph_opt.argtypes = [vp, u64, u32, u32, u32, u32, vp, vp]
            lib.or_seeds_init.argtypes = [u64, u32, u32, u32, vp]
            lib.or_table_address.restype = u32
            lib.or_table_address.argtypes = [vp, u32, u32, u32, u32]
            lib.or_mix31.restype = u32
            lib.or_mix31.argtypes = [u32]
            lib.or_priority.restype = u32
            lib.or_priority.argtypes = [u32, u32]
            lib.or_cm_cell.restype = u32
            lib.or_cm_cell.argtypes = [u32, u32, u32]
            lib.or_hash_rows.argtypes = [u32, u32, u32, u32, vp, vp, vp, u64, vp, vp]
            lib.or_new.restype = vp
            lib.or_new.argtypes = [u32, u32, u32, u32, u32, u32, u32, u64, u64, u32]
            lib.or_new_partial.restype = vp
            lib.or_new_partial.argtypes = [u32, u32, u32, u32, u32, u32, u32, u64, u64, vp, vp, u64, u32]
            lib.or_free.argtypes = [vp]
            lib.or_seeds.restype = ctypes.POINTER(u32)
            lib.or_seeds.argtypes = [vp]
            lib.or_insert.restype = i32
            lib.or_insert.argtypes = [vp, vp, vp, u64, ctypes.POINTER(u64)]
            lib.or_insert_parallel.restype = i32
            lib.or_insert_parallel.argtypes = [vp, vp, vp, u64, ctypes.POINTER(u64), i32]
            lib.or_bucket.restype = i32
            lib.or_bucket.argtypes = [vp, u32, u32, u32, vp, vp]
            lib.or_export.restype = i32
            lib.or_export.argtypes = [vp, vp, vp]
            lib.or_query_one.restype = i32
            lib.or_query_one.argtypes = [vp, vp, u64, u32, vp, vp, vp, ctypes.POINTER(u64), vp,
                                         ctypes.POINTER(u64), vp, vp, vp]
            lib.or_query.restype = i32
            lib.or_query.argtypes = [vp, vp, vp, u64, u32, vp, vp]
            lib.or_next_id.restype = u64
            lib.or_next_id.argtypes = [vp]
            lib.or_jaccard_topk.restype = i32
            lib.or_jaccard_topk.argtypes = [vp, vp, u64, u32, vp, vp, u64, u32, i32, vp, vp, vp]
            lib.or_set_next_id.restype = i32
            lib.or_set_next_id.argtypes = [vp, u64]
            lib.or_tk_update.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), u32]
            lib.or_tk_merge_cell.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), u32, u32]
            lib.or_tk_new.restype = vp
            lib.or_tk_new.argtypes = [u32, u32, u32, u32, u32, u32, u64, u64, u32]
            lib.or_tk_free.argtypes = [vp]
            lib.or_tk_insert.restype = i32
            lib.or_tk_insert.argtypes = [vp, vp, vp, u64, ctypes.POINTER(u64)]
            lib.or_tk_export.argtypes = [vp, vp]
            lib.or_tk_new_partial.restype = vp
            lib.or_tk_new_partial.argtypes = [u32, u32, u32, u32, u32, u32, u64, u64, u32, vp, vp, u64]
            lib.or_tk_insert_parallel.restype = i32
            lib.or_tk_insert_parallel.argtypes = [vp, vp, vp, u64, ctypes.POINTER(u64), i32]
            lib.or_tk_bucket.restype = i32
            lib.or_tk_bucket.argtypes = [vp, u32, u32, u32, vp]
            lib.or_tk_query.restype = i32
            lib.or_tk_query.argtypes = [vp, vp, vp, u64, u32, u32, vp, vp]
            lib.or_tk_fold.argtypes = [vp, vp, u64, u32, vp, vp]
            lib.or_tk_rank.argtypes = [vp, vp, u32, u32, u32, vp, vp]
            _lib = lib
    return _lib


def _p(a: np.ndarray | None) -> int | None:
    return None if a is None else a.ctypes.data


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


# ---------------------------------------------------------------- primitives
def mix32(x: int) -> int:
    return int(_load().or_mix32(x & 0xFFFFFFFF))


def splitmix64_stream(seed: int, n: int) -> list[int]:
    st = ctypes.c_uint64(seed)
    lib = _load()
    return [int(lib.or_splitmix64_next(ctypes.byref(st))) for _ in range(n)]


def derive_seeds(seed: int, L: int, d: int) -> dict:
    out = np.empty(2 + 2 * L + d, dtype=np.uint32)
    _load().or_derive_seeds(seed, L, d, _p(out))
    return {"a": int(out[0]), "dirseed": int(out[1]), "st": out[2:2 + L].copy(),
            "sp": out[2 + L:2 + 2 * L].copy(), "sc": out[2 + 2 * L:].copy(), "raw": out}


def minhash(cols, a: int) -> int:
    c = _u32(cols)
    return int(_load().or_minhash(_p(c), c.size, a))


def doph(cols, nb: int, a: int, dirseed: int) -> tuple[np.ndarray, np.ndarray]:
    """DOPH codes[nb] and the pre-densification non-empty mask[nb]."""
    c = _u32(cols)
    codes = np.empty(nb, dtype=np.uint32)
    mask = np.empty(nb, dtype=np.uint8)
    _load().or_doph(_p(c), c.size, nb, a, dirseed, _p(codes), _p(mask))
    return codes, mask.astype(bool)


def doph_opt(cols, nb: int, a: int, od: int, dirseed: int) -> tuple[np.ndarray, np.ndarray]:
    """DOPH with optimal densification: codes[nb] and the non-empty mask[nb]."""
    c = _u32(cols)
    codes = np.empty(nb, dtype=np.uint32)
    mask = np.empty(nb, dtype=np.uint8)
    _load().or_doph_opt(_p(c), c.size, nb, a, od, dirseed, _p(codes), _p(mask))
    return codes, mask.astype(bool)


def seeds_init(seed: int, L: int, d: int, densify: int = 0) -> np.ndarray:
    """The index's seed words: derive_seeds' words, od, the densification mode."""
    out = np.empty(2 + 2 * L + d + 2, dtype=np.uint32)
    _load().or_seeds_init(seed, L, d, densify, _p(out))
    return out


def table_address(codes, t: int, K: int, B: int, st_t: int) -> int:
    c = _u32(codes)
    return int(_load().or_table_address(_p(c), t, K, B, st_t))


def mix31(x: int) -> int:
    return int(_load().or_mix31(x & 0xFFFFFFFF))


def priority(id_: int, sp_t: int) -> int:
    return int(_load().or_priority(id_, sp_t))


def cm_cell(id_: int, sc_r: int, w: int) -> int:
    return int(_load().or_cm_cell(id_, sc_r, w))


def hash_rows(K: int, L: int, B: int, seed: int, d: int, offs, cols, want_codes: bool = True,
              densify: int = 0):
    """Codes [n][K*L] (or None) and table addresses [n][L] for CSR rows."""
    offs, cols = _u64(offs), _u32(cols)
    n = offs.size - 1
    s = seeds_init(seed, L, d, densify)
    codes = np.empty((n, K * L), dtype=np.uint32) if want_codes else None
    bk = np.empty((n, L), dtype=np.uint32)
    _load().or_hash_rows(K, L, B, d, _p(s), _p(offs), _p(cols), n, _p(codes), _p(bk))
    return codes, bk


# ---------------------------------------------------------------- index
class Index:
    """Oracle index.  Dense by default; ``partial=(req_t, req_b)`` keeps only the
    listed buckets (bounded memory for full-size sampled checks)."""

    def __init__(self, *, K: int, L: int, log2_buckets: int, reservoir: int, cm_rows: int,
                 cm_width: int, shards: int = 1, seed: int = 0, capacity: int, partial=None,
                 densify: int = 0):
        self._lib = _load()
        self.K, self.L, self.B, self.R = K, L, log2_buckets, reservoir
        self.d, self.w, self.S, self.capacity = cm_rows, cm_width, shards, capacity
        if partial is None:
            self._h = self._lib.or_new(K, L, log2_buckets, reservoir, cm_rows, cm_width, shards,
                                       seed, capacity, densify)
        else:
            rt, rb = _u32(partial[0]), _u32(partial[1])
            self._h = self._lib.or_new_partial(K, L, log2_buckets, reservoir, cm_rows, cm_width,
                                               shards, seed, capacity, _p(rt), _p(rb), rt.size, densify)
        if not self._h:
            raise MemoryError("oracle index allocation failed")
        self.partial = partial is not None

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.or_free(h)

    @property
    def next_id(self) -> int:
        return int(self._lib.or_next_id(self._h))

    def set_next_id(self, id_: int) -> None:
        """Rows inserted next take ids from id_ on (a partition starting at its global id)."""
        if self._lib.or_set_next_id(self._h, id_):
            raise ValueError("next id must not go back nor pass the capacity")

    def insert(self, offs, cols, threads: int = 1) -> int:
        offs, cols = _u64(offs), _u32(cols)
        first = ctypes.c_uint64()
        if threads > 1 and self.partial:
            rc = self._lib.or_insert_parallel(self._h, _p(offs), _p(cols), offs.size - 1,
                                              ctypes.byref(first), threads)
        else:
            rc = self._lib.or_insert(self._h, _p(offs), _p(cols), offs.size - 1, ctypes.byref(first))
        if rc:
            raise ValueError(f"oracle insert failed ({rc}): capacity exceeded")
        return int(first.value)

    def bucket(self, t: int, b: int, s: int = 0) -> tuple[np.ndarray, int]:
        slots = np.empty(self.R, dtype=np.uint32)
        fill = ctypes.c_uint32()
        if self._lib.or_bucket(self._h, s, t, b, _p(slots), ctypes.byref(fill)):
            raise KeyError((t, b))
        return slots, int(fill.value)

    def export(self) -> tuple[np.ndarray, np.ndarray]:
        """slots [S][L][2^B][R] and fill [S][L][2^B] (dense index only)."""
        nb = self.S * (self.L << self.B)
        slots = np.empty(nb * self.R, dtype=np.uint32)
        fill = np.empty(nb, dtype=np.uint32)
        if self._lib.or_export(self._h, _p(slots), _p(fill)):
            raise ValueError("export needs a dense index")
        return (slots.reshape(self.S, self.L, 1 << self.B, self.R),
                fill.reshape(self.S, self.L, 1 << self.B))

    def query(self, offs, cols, k: int) -> tuple[np.ndarray, np.ndarray]:
        offs, cols = _u64(offs), _u32(cols)
        nq = offs.size - 1
        ids = np.empty((nq, k), dtype=np.int32)
        scores = np.empty((nq, k), dtype=np.uint32)
        if self._lib.or_query(self._h, _p(offs), _p(cols), nq, k, _p(ids), _p(scores)):
            raise KeyError("query touched a bucket the partial index does not hold")
        return ids, scores

    def query_detail(self, cols, k: int) -> dict:
        """One query with its candidate multiset, distinct ids, estimates, exact counts, sketch."""
        c = _u32(cols)
        cap = self.S * self.L * self.R
        ids = np.empty(k, dtype=np.int32)
        scores = np.empty(k, dtype=np.uint32)
        M = np.empty(cap + 1, dtype=np.uint32)
        U = np.empty(cap + 1, dtype=np.uint32)
        est = np.empty(cap + 1, dtype=np.uint32)
        cnt = np.empty(cap + 1, dtype=np.uint32)
        cm = np.empty(self.d * self.w, dtype=np.uint32)
        ml, ul = ctypes.c_uint64(), ctypes.c_uint64()
        rc = self._lib.or_query_one(self._h, _p(c), c.size, k, _p(ids), _p(scores), _p(M),
                                    ctypes.byref(ml), _p(U), ctypes.byref(ul), _p(est), _p(cnt),
                                    _p(cm))
        if rc:
            raise KeyError("query touched a bucket the partial index does not hold")
        m, u = int(ml.value), int(ul.value)
        return {"ids": ids, "scores": scores, "M": M[:m].copy(), "U": U[:u].copy(),
                "est": est[:u].copy(), "cnt": cnt[:u].copy(), "cm": cm.reshape(self.d, self.w)}


# ---------------------------------------------------------------- TopKAPI buckets
def tk_update(cell: tuple[int, int], x: int) -> tuple[int, int]:
    """One Appendix 2 insertion into a (heavy hitter, count) cell."""
    h, c = ctypes.c_uint32(cell[0]), ctypes.c_uint32(cell[1])
    _load().or_tk_update(ctypes.byref(h), ctypes.byref(c), x)
    return int(h.value), int(c.value)


def tk_merge(a: tuple[int, int], b: tuple[int, int]) -> tuple[int, int]:
    """Appendix 2 merge of two cells (count 0 = empty)."""
    h, c = ctypes.c_uint32(a[0]), ctypes.c_uint32(a[1])
    _load().or_tk_merge_cell(ctypes.byref(h), ctypes.byref(c), b[0], b[1])
    return int(h.value), int(c.value)


def jaccard_topk(offs, cols, qoffs, qcols, k: int, dim: int = 1 << 20, threads: int = 1):
    """Exact Jaccard top-k of every query over the collection (brute force):
    (ids [nq][k] (-1 pad), intersections, unions) ranked (similarity desc, id asc)."""
    offs, cols, qoffs, qcols = _u64(offs), _u32(cols), _u64(qoffs), _u32(qcols)
    nq = qoffs.size - 1
    ids = np.empty((nq, k), np.int32)
    inter = np.empty((nq, k), np.uint32)
    uni = np.empty((nq, k), np.uint32)
    _load().or_jaccard_topk(_p(offs), _p(cols), offs.size - 1, dim, _p(qoffs), _p(qcols), nq, k, threads, _p(ids),
                            _p(inter), _p(uni))
    return ids, inter, uni


def tk_fold(sketches) -> tuple[np.ndarray, np.ndarray]:
    """Appendix 2 merge of a sequence of sketches, in the given order, into an
    empty sketch.  ``sketches``: [n][cells][2] (heavy hitter, count) pairs;
    returns (heavy hitters, counts) of the merged cells."""
    a = np.ascontiguousarray(sketches, dtype=np.uint32)
    n, wc = a.shape[0], a.shape[1]
    hh, cnt = np.ascontiguousarray(a[..., 0]), np.ascontiguousarray(a[..., 1])
    mh, mc = np.empty(wc, np.uint32), np.empty(wc, np.uint32)
    _load().or_tk_fold(_p(hh), _p(cnt), n, wc, _p(mh), _p(mc))
    return mh, mc


def tk_rank(mh, mc, k: int, threshold: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Appendix 2 query report of one merged sketch: top-k (ids, scores)."""
    mh, mc = _u32(mh), _u32(mc)
    ids, scores = np.empty(k, np.int32), np.empty(k, np.uint32)
    _load().or_tk_rank(_p(mh), _p(mc), mh.size, k, threshold, _p(ids), _p(scores))
    return ids, scores


class TkIndex:
    """Oracle index whose buckets are TopKAPI sketches of W rows x C cells."""

    def __init__(self, *, K: int, L: int, log2_buckets: int, rows: int, cells: int, shards: int = 1,
                 seed: int = 0, capacity: int, densify: int = 0, partial=None):
        self._lib = _load()
        self.K, self.L, self.B, self.W, self.C, self.S = K, L, log2_buckets, rows, cells, shards
        if partial is None:
            self._h = self._lib.or_tk_new(K, L, log2_buckets, rows, cells, shards, seed, capacity, densify)
        else:
            rt, rb = _u32(partial[0]), _u32(partial[1])
            self._h = self._lib.or_tk_new_partial(K, L, log2_buckets, rows, cells, shards, seed, capacity,
                                                  densify, _p(rt), _p(rb), rt.size)
        if not self._h:
            raise MemoryError("oracle sketch allocation failed")
        self.partial = partial is not None

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.or_tk_free(h)

    def insert(self, offs, cols, threads: int = 1) -> int:
        offs, cols = _u64(offs), _u32(cols)
        first = ctypes.c_uint64()
        if threads > 1:
            rc = self._lib.or_tk_insert_parallel(self._h, _p(offs), _p(cols), offs.size - 1, ctypes.byref(first),
                                                 threads)
        else:
            rc = self._lib.or_tk_insert(self._h, _p(offs), _p(cols), offs.size - 1, ctypes.byref(first))
        if rc:
            raise ValueError("oracle insert failed: capacity exceeded")
        return int(first.value)

    def bucket(self, t: int, b: int, s: int = 0) -> np.ndarray:
        """cells [W][C][2] of sketch (s, t, b) = (heavy hitter or EMPTY, count)."""
        out = np.empty((self.W, self.C, 2), dtype=np.uint32)
        if self._lib.or_tk_bucket(self._h, s, t, b, _p(out)):
            raise KeyError((s, t, b))
        return out

    def export(self) -> np.ndarray:
        """cells [S][L][2^B][W][C][2] = (heavy hitter or EMPTY, count)."""
        out = np.empty((self.S, self.L, 1 << self.B, self.W, self.C, 2), dtype=np.uint32)
        self._lib.or_tk_export(self._h, _p(out))
        return out

    def query(self, offs, cols, k: int, threshold: int = 0):
        """Top-k heavy hitters of the merged sketch whose count exceeds ``threshold``."""
        offs, cols = _u64(offs), _u32(cols)
        nq = offs.size - 1
        ids = np.empty((nq, k), dtype=np.int32)
        scores = np.empty((nq, k), dtype=np.uint32)
        if self._lib.or_tk_query(self._h, _p(offs), _p(cols), nq, k, threshold, _p(ids), _p(scores)):
            raise KeyError("a query's sketch is not kept by this partial index")
        return ids, scores

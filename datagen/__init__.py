"""Seeded synthetic inputs (CSR rows and queries) for the SLASH hot path.

Inputs only: nothing here hashes, buckets or counts.  The oracle (CPU) and the
CUDA path both consume these arrays.  The generator itself is plain C
(``slashgen.c``) loaded with ctypes; it is compiled in place on first use.

Workload shape (synthetic stand-in for the Criteo click logs of the paper's
evaluation, Sec. 6): 2^20 hashed binary features, ~40 non-zeros per row,
Zipf(1.1) feature popularity.  See ``workloads.py`` for the named sizes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slashgen.c")
_LIB = os.path.join(_HERE, "libslashgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libslashgen.so`` next to its source (gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32, u64, i32, dbl, vp = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p)
            lib.sg_new.restype = vp
            lib.sg_new.argtypes = [u32, dbl, dbl, dbl, dbl, u32]
            lib.sg_free.argtypes = [vp]
            lib.sg_rows_nnz.argtypes = [vp, u64, u64, u64, u32, u32, vp, i32]
            lib.sg_rows_cols.argtypes = [vp, u64, u64, u64, vp, vp, i32]
            lib.sg_queries_meta.argtypes = [vp, u64, u64, u64, u64, u64, u32, u32, dbl, u32, u32,
                                            vp, vp, i32]
            lib.sg_queries_cols.argtypes = [vp, u64, u64, u64, u64, dbl, vp, vp, vp, i32]
            lib.sg_zipf_cdf.restype = ctypes.POINTER(ctypes.c_uint64)
            lib.sg_zipf_cdf.argtypes = [vp]
            lib.sg_pois_cdf.restype = ctypes.POINTER(ctypes.c_uint64)
            lib.sg_pois_cdf.argtypes = [vp, ctypes.POINTER(u32)]
            lib.sg_lnorm_cdf.restype = ctypes.POINTER(ctypes.c_uint64)
            lib.sg_lnorm_cdf.argtypes = [vp, ctypes.POINTER(u32)]
            lib.sg_zipf_guide.restype = ctypes.POINTER(u32)
            lib.sg_zipf_guide.argtypes = [vp]
            lib.sg_pois_guide.restype = ctypes.POINTER(u32)
            lib.sg_pois_guide.argtypes = [vp]
            lib.sg_feature.restype = u32
            lib.sg_feature.argtypes = [vp, u64, u64]
            lib.sg_u64_public.restype = u64
            lib.sg_u64_public.argtypes = [u64, u32, u64, u32]
            _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Generator:
    """Seeded generator of sparse binary rows over ``2**dim_bits`` features."""

    def __init__(self, dim_bits: int = 20, zipf_s: float = 1.1, pois_lambda: float = 40.0,
                 ln_mu: float = math.log(40.0), ln_sigma: float = 1.0, ln_max: int = 2000):
        self._lib = _load()
        self._h = self._lib.sg_new(dim_bits, zipf_s, pois_lambda, ln_mu, ln_sigma, ln_max)
        if not self._h:
            raise ValueError("invalid generator parameters (dim_bits must be even, 2..30)")
        self.dim_bits = dim_bits
        self.dim = 1 << dim_bits
        self.ln_max = ln_max

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.sg_free(h)

    # -- tables (for tests and for other generators that reuse them) --
    def zipf_cdf(self) -> np.ndarray:
        p = self._lib.sg_zipf_cdf(self._h)
        return np.ctypeslib.as_array(p, shape=(self.dim,)).copy()

    def poisson_cdf(self) -> np.ndarray:
        n = ctypes.c_uint32()
        p = self._lib.sg_pois_cdf(self._h, ctypes.byref(n))
        return np.ctypeslib.as_array(p, shape=(n.value,)).copy()

    def lognormal_cdf(self) -> np.ndarray:
        n = ctypes.c_uint32()
        p = self._lib.sg_lnorm_cdf(self._h, ctypes.byref(n))
        return np.ctypeslib.as_array(p, shape=(n.value,)).copy()

    def zipf_guide(self) -> np.ndarray:
        return np.ctypeslib.as_array(self._lib.sg_zipf_guide(self._h), shape=(65537,)).copy()

    def poisson_guide(self) -> np.ndarray:
        return np.ctypeslib.as_array(self._lib.sg_pois_guide(self._h), shape=(65537,)).copy()

    def feature(self, seed: int, u: int) -> int:
        return int(self._lib.sg_feature(self._h, seed, u))

    # -- rows --
    def rows_nnz(self, seed: int, row0: int, n: int, lo: int = 5, hi: int = 200,
                 threads: int | None = None) -> np.ndarray:
        nnz = np.empty(n, dtype=np.uint32)
        if n:
            self._lib.sg_rows_nnz(self._h, seed, row0, n, lo, hi, _ptr(nnz),
                                  threads or default_threads())
        return nnz

    def rows(self, seed: int, row0: int, n: int, lo: int = 5, hi: int = 200,
             threads: int | None = None) -> tuple[np.ndarray, np.ndarray]:
        """Rows ``[row0, row0+n)`` as CSR: ``offs`` uint64[n+1] (from 0), ``cols`` uint32."""
        nnz = self.rows_nnz(seed, row0, n, lo, hi, threads)
        offs = np.zeros(n + 1, dtype=np.uint64)
        np.cumsum(nnz, out=offs[1:])
        cols = np.empty(int(offs[-1]), dtype=np.uint32)
        if n:
            self._lib.sg_rows_cols(self._h, seed, row0, n, _ptr(offs), _ptr(cols),
                                   threads or default_threads())
        return offs, cols

    # -- queries --
    def queries(self, seed: int, qseed: int, nq: int, n_rows: int, *, lo: int = 5, hi: int = 200,
                planted_frac: float = 1.0, p_perturb: float = 0.2, rlo: int = 1, rhi: int = 2000,
                q0: int = 0, threads: int | None = None):
        """Queries ``[q0, q0+nq)``: planted (perturbed dataset rows) or random lognormal rows.

        Returns ``(offs, cols, src)``; ``src[i]`` is the planted source row or -1.
        """
        src = np.empty(nq, dtype=np.int64)
        nnz = np.empty(nq, dtype=np.uint32)
        t = threads or default_threads()
        if nq:
            self._lib.sg_queries_meta(self._h, seed, qseed, q0, nq, n_rows, lo, hi,
                                      planted_frac, rlo, rhi, _ptr(src), _ptr(nnz), t)
        offs = np.zeros(nq + 1, dtype=np.uint64)
        np.cumsum(nnz, out=offs[1:])
        cols = np.empty(int(offs[-1]), dtype=np.uint32)
        if nq:
            self._lib.sg_queries_cols(self._h, seed, qseed, q0, nq, p_perturb, _ptr(src),
                                      _ptr(offs), _ptr(cols), t)
        return offs, cols, src


def u64(seed: int, stream: int, row: int, j: int) -> int:
    """The generator's counter-based uniform word (exposed for tests)."""
    return int(_load().sg_u64_public(seed, stream, row, j))


# ---------------------------------------------------------------------- device twin
_DEV_SRC = os.path.join(_HERE, "slashgen_dev.cu")
_DEV_LIB = os.path.join(_HERE, "libslashgen_dev.so")
_dev_lib = None


def build_device(force: bool = False) -> str:
    """Compile the CUDA twin (sm_103a) next to its source."""
    if force or not os.path.exists(_DEV_LIB) or os.path.getmtime(_DEV_LIB) < os.path.getmtime(_DEV_SRC):
        tmp = _DEV_LIB + f".tmp{os.getpid()}"
        nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3",
                               "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _DEV_SRC])
        os.replace(tmp, _DEV_LIB)
    return _DEV_LIB


def _load_dev():
    global _dev_lib
    with _lock:
        if _dev_lib is None:
            lib = ctypes.CDLL(build_device())
            vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
            lib.sgd_rows_nnz.restype = ctypes.c_int
            lib.sgd_rows_nnz.argtypes = [vp, vp, u32, u64, u64, u32, u32, u32, u32, vp, vp]
            lib.sgd_rows_cols.restype = ctypes.c_int
            lib.sgd_rows_cols.argtypes = [vp, vp, u32, u64, u64, u32, vp, vp, vp]
            _dev_lib = lib
    return _dev_lib


class DeviceRows:
    """Dataset rows generated on the GPU, byte-identical to ``Generator.rows``."""

    def __init__(self, gen: Generator, device: str = "cuda"):
        import torch
        self.torch = torch
        self._lib = _load_dev()
        self.dim_bits, self.dim = gen.dim_bits, gen.dim
        t = lambda a, dt: torch.from_numpy(a.view(dt)).to(device)
        self.zc = t(gen.zipf_cdf(), np.int64)
        self.zg = t(gen.zipf_guide(), np.int32)
        pc = gen.poisson_cdf()
        self.pn = len(pc)
        self.pc = t(pc, np.int64)
        self.pg = t(gen.poisson_guide(), np.int32)
        self.device = device

    def rows(self, seed: int, row0: int, n: int, lo: int = 5, hi: int = 200, stream=None):
        """(offs int64 [n+1] from 0, cols int32) CUDA tensors for rows [row0, row0+n)."""
        torch = self.torch
        st = stream or torch.cuda.current_stream()
        with torch.cuda.stream(st):
            nnz = torch.empty(n, dtype=torch.int32, device=self.device)
            rc = self._lib.sgd_rows_nnz(self.pc.data_ptr(), self.pg.data_ptr(), self.pn, seed, row0, n, lo, hi,
                                        self.dim, nnz.data_ptr(), st.cuda_stream)
            if rc:
                raise RuntimeError("device generator launch failed")
            offs = torch.zeros(n + 1, dtype=torch.int64, device=self.device)
            torch.cumsum(nnz, 0, out=offs[1:])
            total = int(offs[-1].item())
            cols = torch.empty(total, dtype=torch.int32, device=self.device)
            rc = self._lib.sgd_rows_cols(self.zc.data_ptr(), self.zg.data_ptr(), self.dim_bits, seed, row0, n,
                                         offs.data_ptr(), cols.data_ptr(), st.cuda_stream)
            if rc:
                raise RuntimeError("device generator launch failed")
        return offs, cols

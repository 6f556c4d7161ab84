"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point its header declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(slash_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_four_calls():
    names = _declared()
    for n in ("slash_build_index", "slash_insert", "slash_query", "slash_free",
              "slash_tk_build", "slash_tk_insert", "slash_tk_query", "slash_tk_free"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2008_03260_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (slash_\w+)", out))
    assert set(_declared()) <= exported


def test_strerror_without_gpu():
    from paper_2008_03260_b300 import build
    lib = ctypes.CDLL(build.build())
    lib.slash_strerror.restype = ctypes.c_char_p
    assert lib.slash_strerror(0) == b"ok"
    assert lib.slash_strerror(-4) == b"index capacity exceeded"


def test_build_index_rejects_bad_params_without_touching_the_gpu():
    """Parameter validation happens before any CUDA call."""
    import paper_2008_03260_b300 as s
    bad = [dict(L=0), dict(L=200), dict(K=64, L=64), dict(cm_width=1000), dict(reservoir=0),
           dict(capacity=1 << 31), dict(log2_buckets=0), dict(cm_rows=9), dict(shards=65)]
    for b in bad:
        p = s.Params(**b)
        h = ctypes.c_void_p()
        rc = s._lib.slash_build_index(ctypes.byref(p.c()), None, ctypes.byref(h))
        assert rc == s.SLASH_EINVAL, b
        assert h.value is None


def test_checkpoint_file_errors_without_gpu(tmp_path):
    """slash_load checks the file before it touches a device."""
    from paper_2008_03260_b300 import build
    lib = ctypes.CDLL(build.build())
    out = ctypes.c_void_p()
    missing = str(tmp_path / "missing.ix").encode()
    assert lib.slash_load(missing, None, ctypes.byref(out)) == -8       # SLASH_EIO
    assert lib.slash_tk_load(missing, None, ctypes.byref(out)) == -8
    junk = tmp_path / "junk.ix"
    junk.write_bytes(b"NOTSLASH" + b"\0" * 200)
    assert lib.slash_load(str(junk).encode(), None, ctypes.byref(out)) == -1   # SLASH_EINVAL
    assert lib.slash_tk_load(str(junk).encode(), None, ctypes.byref(out)) == -1
    assert out.value is None


def test_set_allocator_validates_without_gpu():
    import ctypes

    import paper_2008_03260_b300 as s
    none_a, none_f = s.SLASH_ALLOC_FN(), s.SLASH_FREE_FN()
    assert s._lib.slash_set_allocator(None, none_a, none_f, None) == s.SLASH_EINVAL      # no index
    only_alloc = s.SLASH_ALLOC_FN(lambda n, c: None)
    assert s._lib.slash_set_allocator(ctypes.c_void_p(1), only_alloc, none_f, None) == s.SLASH_EINVAL
    only_free = s.SLASH_FREE_FN(lambda p, c: None)
    assert s._lib.slash_set_allocator(ctypes.c_void_p(1), none_a, only_free, None) == s.SLASH_EINVAL

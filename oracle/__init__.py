"""CPU oracle for exact multi-pattern search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the GPU
library (``paper_1704_02278_gb300``) and the GPU library never imports it.

The arithmetic lives in ``glop_oracle.c`` (plain C, built with gcc):

* :func:`naive`   -- every pattern compared at every offset (the naive
  approach of Sec. 2).
* :func:`ac`      -- the Aho-Corasick automaton of Sec. 4 (goto graph, failure
  function by BFS, output(s) = own(s) U output(fail(s))), one pass, matches
  converted from end to start position and sorted.
* :func:`ac_mt`   -- the chunked multi-threaded Aho-Corasick of Sec. 4, chunks
  overlapping by (longest pattern - 1) bytes.
* :func:`batch`   -- the same definition per segment of a concatenated buffer.
* :func:`ac_trace` -- goto/failure transitions on a text (worked example of
  Sec. 4).

Every function takes ``prefix_len``: 0 is exact full-pattern matching; K > 0
cuts every pattern to its first K bytes first (prefix matching, Sec. 1/5).
Results are ``(M, 2)`` uint32 arrays of (offset, pattern_id) sorted by
(offset, pattern_id), or ``(M, 3)`` (segment, offset, pattern_id) for batch.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glop_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False, extra_flags=(), out_path: str | None = None) -> str:
    """Compile ``glop_oracle.c`` into a shared library with gcc; returns its path."""
    out = out_path or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", *extra_flags, _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    u32pp = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))
    for name in ("oracle_naive", "oracle_ac", "oracle_kmp"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [u8p, ctypes.c_uint64, u8p, u64p, ctypes.c_uint32, ctypes.c_uint32, u32pp, u64p]
    lib.oracle_ac_mt.restype = ctypes.c_int
    lib.oracle_ac_mt.argtypes = [u8p, ctypes.c_uint64, u8p, u64p, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_uint32, u32pp, u64p]
    lib.oracle_batch.restype = ctypes.c_int
    lib.oracle_batch.argtypes = [u8p, u64p, ctypes.c_uint32, u8p, u64p, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_int, ctypes.c_uint32, u32pp, u64p]
    lib.oracle_ac_trace.restype = ctypes.c_int64
    lib.oracle_ac_trace.argtypes = [u8p, ctypes.c_uint64, u8p, u64p, ctypes.c_uint32, ctypes.c_char_p,
                                    ctypes.c_uint64]
    lib.oracle_free.restype = None
    lib.oracle_free.argtypes = [ctypes.c_void_p]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  ``path`` loads another build (tests)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class OracleError(RuntimeError):
    def __init__(self, rc: int):
        super().__init__({1: "invalid argument", 2: "out of memory"}.get(rc, "error %d" % rc))
        self.rc = rc


def pattern_csr(patterns):
    """``patterns`` as (uint8 bytes, uint64 offsets[n+1]); accepts a list of bytes or such a tuple."""
    if isinstance(patterns, tuple) and len(patterns) == 2:
        buf = np.ascontiguousarray(patterns[0], dtype=np.uint8)
        offs = np.ascontiguousarray(patterns[1], dtype=np.uint64)
        return buf, offs
    pats = [bytes(p) for p in patterns]
    offs = np.zeros(len(pats) + 1, dtype=np.uint64)
    if pats:
        offs[1:] = np.cumsum([len(p) for p in pats])
    buf = np.frombuffer(b"".join(pats), dtype=np.uint8) if pats else np.zeros(0, np.uint8)
    return np.ascontiguousarray(buf), offs


def _as_u8(text):
    if isinstance(text, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(text), dtype=np.uint8)
    return np.ascontiguousarray(text, dtype=np.uint8).reshape(-1)


def _ptr(a, ct):
    if a.size == 0:
        # a valid non-null pointer for empty arrays
        a = np.zeros(1, dtype=a.dtype)
        _ptr.keep.append(a)
    return a.ctypes.data_as(ctypes.POINTER(ct))


_ptr.keep = []


def _take(lib, outp, count, width):
    n = int(count.value) * width
    if n == 0:
        if outp:
            lib.oracle_free(outp)
        return np.zeros((0, width), dtype=np.uint32)
    arr = np.ctypeslib.as_array(outp, shape=(n,)).copy().reshape(-1, width)
    lib.oracle_free(outp)
    return arr


class Oracle:
    """The oracle functions bound to one build of ``glop_oracle.c``."""

    def __init__(self, lib):
        self.lib = lib

    def _run(self, fn_name, text, patterns, prefix_len, *extra):
        lib = self.lib
        t = _as_u8(text)
        buf, offs = pattern_csr(patterns)
        outp = ctypes.POINTER(ctypes.c_uint32)()
        count = ctypes.c_uint64(0)
        npat = len(offs) - 1
        rc = getattr(lib, fn_name)(_ptr(t, ctypes.c_uint8), t.size, _ptr(buf, ctypes.c_uint8),
                                   _ptr(offs, ctypes.c_uint64), npat, int(prefix_len), *extra,
                                   ctypes.byref(outp), ctypes.byref(count))
        _ptr.keep.clear()
        if rc:
            raise OracleError(rc)
        return _take(lib, outp, count, 2)

    def naive(self, text, patterns, prefix_len: int = 0) -> np.ndarray:
        """Naive scan (Sec. 2): (M, 2) uint32 (offset, pattern_id), sorted."""
        return self._run("oracle_naive", text, patterns, prefix_len)

    def ac(self, text, patterns, prefix_len: int = 0) -> np.ndarray:
        """Single-threaded Aho-Corasick (Sec. 4): (M, 2) uint32 (offset, pattern_id), sorted."""
        return self._run("oracle_ac", text, patterns, prefix_len)

    def ac_mt(self, text, patterns, prefix_len: int = 0, threads: int | None = None) -> np.ndarray:
        """Chunked multi-threaded Aho-Corasick (Sec. 4, overlap = longest pattern - 1)."""
        th = threads or os.cpu_count() or 1
        return self._run("oracle_ac_mt", text, patterns, prefix_len, int(th))

    def kmp(self, text, patterns, prefix_len: int = 0) -> np.ndarray:
        """Knuth-Morris-Pratt once per pattern (Sec. 2, Sec. 7): (M, 2) uint32 (offset, pattern_id), sorted."""
        return self._run("oracle_kmp", text, patterns, prefix_len)

    def batch(self, text, seg_offsets, patterns, prefix_len: int = 0, method: str = "ac",
              threads: int | None = None) -> np.ndarray:
        """Per-segment definition: (M, 3) uint32 (segment, offset-in-segment, pattern_id), sorted."""
        lib = self.lib
        t = _as_u8(text)
        seg = np.ascontiguousarray(seg_offsets, dtype=np.uint64)
        buf, offs = pattern_csr(patterns)
        outp = ctypes.POINTER(ctypes.c_uint32)()
        count = ctypes.c_uint64(0)
        th = threads or os.cpu_count() or 1
        rc = lib.oracle_batch(_ptr(t, ctypes.c_uint8), _ptr(seg, ctypes.c_uint64), max(len(seg) - 1, 0),
                              _ptr(buf, ctypes.c_uint8), _ptr(offs, ctypes.c_uint64), len(offs) - 1,
                              int(prefix_len), {"naive": 0, "ac": 1}[method], int(th),
                              ctypes.byref(outp), ctypes.byref(count))
        _ptr.keep.clear()
        if rc:
            raise OracleError(rc)
        return _take(lib, outp, count, 3)

    def ac_trace(self, text, patterns) -> str:
        """Goto ("g:") and failure ("f:") transitions per text byte (Sec. 4 worked example)."""
        lib = self.lib
        t = _as_u8(text)
        buf, offs = pattern_csr(patterns)
        cap = 256 * (t.size + 1) + 4096
        out = ctypes.create_string_buffer(cap)
        n = lib.oracle_ac_trace(_ptr(t, ctypes.c_uint8), t.size, _ptr(buf, ctypes.c_uint8),
                                _ptr(offs, ctypes.c_uint64), len(offs) - 1, out, cap)
        _ptr.keep.clear()
        if n < 0:
            raise OracleError(1)
        return out.raw[:n].decode("latin-1")


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(load())
    return _default


def naive(text, patterns, prefix_len: int = 0) -> np.ndarray:
    return default().naive(text, patterns, prefix_len)


def kmp(text, patterns, prefix_len: int = 0) -> np.ndarray:
    return default().kmp(text, patterns, prefix_len)


def ac(text, patterns, prefix_len: int = 0) -> np.ndarray:
    return default().ac(text, patterns, prefix_len)


def ac_mt(text, patterns, prefix_len: int = 0, threads: int | None = None) -> np.ndarray:
    return default().ac_mt(text, patterns, prefix_len, threads)


def batch(text, seg_offsets, patterns, prefix_len: int = 0, method: str = "ac",
          threads: int | None = None) -> np.ndarray:
    return default().batch(text, seg_offsets, patterns, prefix_len, method, threads)


def ac_trace(text, patterns) -> str:
    return default().ac_trace(text, patterns)


def mutant(k: int, directory: str) -> Oracle:
    """Build ``glop_oracle.c`` with planted mistake k (test suite only) and bind it."""
    path = os.path.join(directory, "liboracle_mutant%d.so" % k)
    build(force=True, extra_flags=("-DORACLE_MUTANT=%d" % k,), out_path=path)
    return Oracle(load(path))

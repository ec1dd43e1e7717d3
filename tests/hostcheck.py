"""Loader for the test-only host check of the compiler's tables."""
import ctypes

import numpy as np

from paper_1704_02278_gb300 import _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_hostcheck())
        vp = ctypes.c_void_p
        lib.glop_hostcheck_scan.restype = ctypes.c_int
        lib.glop_hostcheck_scan.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp, vp, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32)),
                                            ctypes.POINTER(ctypes.c_uint64), vp]
        lib.glop_hostcheck_free.argtypes = [vp]
        lib.glop_hostcheck_free.restype = None
        _lib = lib
    return _lib


def scan(text, seg, pat_buf, pat_offs, prefix_len=0, gram_len=0, filter_bits=0):
    """(M, 3) uint32 (segment, offset, pattern_id) and stats dict."""
    lib = _load()
    lib.glop_hostcheck_set_options(ctypes.c_uint32(gram_len), ctypes.c_uint32(filter_bits))
    t = np.ascontiguousarray(text, dtype=np.uint8).reshape(-1)
    if t.size == 0:
        t = np.zeros(1, np.uint8)
    seg = np.ascontiguousarray(seg, dtype=np.uint64)
    pb = np.ascontiguousarray(pat_buf, dtype=np.uint8)
    if pb.size == 0:
        pb = np.zeros(1, np.uint8)
    po = np.ascontiguousarray(pat_offs, dtype=np.uint64)
    out = ctypes.POINTER(ctypes.c_uint32)()
    cnt = ctypes.c_uint64()
    stats = np.zeros(16, np.uint64)
    rc = lib.glop_hostcheck_scan(pb.ctypes.data, po.ctypes.data, len(po) - 1, prefix_len, t.ctypes.data,
                                 seg.ctypes.data, len(seg) - 1, ctypes.byref(out), ctypes.byref(cnt),
                                 stats.ctypes.data)
    if rc:
        raise ValueError("hostcheck rc=%d" % rc)
    n = int(cnt.value) * 3
    if n:
        arr = np.ctypeslib.as_array(out, shape=(n,)).copy().reshape(-1, 3)
        lib.glop_hostcheck_free(out)
    else:
        arr = np.zeros((0, 3), np.uint32)
    keys = ["n_states", "n_dense", "n_classes", "gram_len", "filter_pass", "gram_found", "dense_steps",
            "chain_entries", "chain_bytes", "matched_offsets"]
    return arr, {k: int(stats[i]) for i, k in enumerate(keys)}

"""GB300 multi-pattern scan library -- Python binding of include/glop.h.

Exact multi-pattern search over byte buffers: every (offset, pattern_id) with
pattern ``pattern_id`` equal to ``text[offset : offset + len]``, sorted.  It is
the first searching stage of the paper's GPU log-processing library (Sec. 1:
rules and logs in, the count and locations of suspect events out), done by a
failureless trie walked from every byte offset (Sec. 5) and completed on the
GPU so that every reported match is exact.

This module only marshals arguments: every step of a scan runs in the CUDA
kernels of ``libglop.so``.  PyTorch provides device memory and streams.  There
is no CPU fallback: without the built library or a CUDA device every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["Automaton", "Plan", "GlopError", "lib", "library_path", "STATUS"]

_HERE = os.path.dirname(os.path.abspath(__file__))
# GLOP_LIBRARY selects another build of the library (e.g. the bounds-checked debug build)
_LIB_PATH = os.environ.get("GLOP_LIBRARY") or os.path.join(_HERE, "libglop.so")
_lib = None
_lock = threading.Lock()

STATUS = {0: "GLOP_OK", 1: "GLOP_EINVAL", 2: "GLOP_ENOMEM", 3: "GLOP_EOVERFLOW", 4: "GLOP_ECUDA",
          5: "GLOP_ETIMEOUT", 6: "GLOP_EBUSY", 7: "GLOP_EINTERNAL"}
OK, EINVAL, ENOMEM, EOVERFLOW, ECUDA, ETIMEOUT = 0, 1, 2, 3, 4, 5

# Exported symbols of include/glop.h
SYMBOLS = ["glop_compile", "glop_info_get", "glop_max_pattern_len", "glop_scan_workspace_size", "glop_scan",
           "glop_batch_workspace_size", "glop_scan_batch", "glop_scan_status", "glop_scan_host_staging_size",
           "glop_scan_host", "glop_destroy", "glop_status_str", "glop_scan_noalloc", "glop_plan_create",
           "glop_plan_launch", "glop_plan_destroy", "glop_tune", "glop_batch_split",
           "glop_count_workspace_size", "glop_scan_count", "glop_scan_host_plan", "glop_scan_words",
           "glop_ingest_create", "glop_ingest_feed", "glop_ingest_flush", "glop_ingest_reset", "glop_ingest_info",
           "glop_ingest_destroy", "glop_scan_batch_multi", "glop_batch_multi_kind", "glop_server_create",
           "glop_server_submit", "glop_server_poll", "glop_server_release", "glop_server_stats_get",
           "glop_server_destroy"]


class IngestResult(ctypes.Structure):
    """glop_ingest_result: base stream offset, pointer to count (offset, pattern_id) rows, count."""
    _fields_ = [("base", ctypes.c_uint64), ("matches", ctypes.c_void_p), ("count", ctypes.c_uint64)]


class ServerOpts(ctypes.Structure):
    """glop_server_opts."""
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_batch_requests", ctypes.c_uint32), ("max_batch_bytes", ctypes.c_uint64),
                ("out_rows_per_batch", ctypes.c_uint64), ("fast_bytes", ctypes.c_uint64),
                ("big_bytes", ctypes.c_uint64), ("max_request_bytes", ctypes.c_uint64)]


class ServerResult(ctypes.Structure):
    """glop_server_result: request id, status, pinned (offset, pattern_id) rows, count, completion time."""
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("matches", ctypes.c_void_p),
                ("count", ctypes.c_uint64), ("done_ns", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    """glop_server_stats."""
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "batches", "fast", "big", "rescans", "admission_waits",
                                                "requests_per_batch_max", "sets_per_batch_max", "pending",
                                                "inflight", "pinned_allocs")]


class GlopError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__("%s%s" % (STATUS.get(code, "status %d" % code), (": " + what) if what else ""))
        self.code = code


class glop_compile_opts(ctypes.Structure):
    _fields_ = [("prefix_len", ctypes.c_uint32), ("smem_budget_bytes", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("gram_len", ctypes.c_uint32), ("filter_bits_log2", ctypes.c_uint32),
                ("chunk_subtiles", ctypes.c_uint32)]


class glop_tune_point(ctypes.Structure):
    _fields_ = [("opts", glop_compile_opts), ("gbps", ctypes.c_double)]


class glop_info(ctypes.Structure):
    _fields_ = [("n_patterns", ctypes.c_uint32), ("min_pattern_len", ctypes.c_uint32),
                ("max_pattern_len", ctypes.c_uint32), ("n_states", ctypes.c_uint32),
                ("n_dense_states", ctypes.c_uint32), ("n_chain_states", ctypes.c_uint32),
                ("n_classes", ctypes.c_uint32), ("gram_len", ctypes.c_uint32), ("n_grams", ctypes.c_uint32),
                ("cum_ids", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64), ("compile_ms", ctypes.c_double)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """The loaded libglop.so; raises if it was not built (run ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libglop.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
        L = ctypes.CDLL(_LIB_PATH)
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.glop_compile.restype = ctypes.c_int
        L.glop_compile.argtypes = [vp, vp, u32, ctypes.POINTER(glop_compile_opts), ctypes.POINTER(vp)]
        L.glop_info_get.restype = ctypes.c_int
        L.glop_info_get.argtypes = [vp, ctypes.POINTER(glop_info)]
        L.glop_max_pattern_len.restype = u32
        L.glop_max_pattern_len.argtypes = [vp]
        L.glop_scan_workspace_size.restype = ctypes.c_int
        L.glop_scan_workspace_size.argtypes = [vp, u64, ctypes.POINTER(u64)]
        L.glop_batch_workspace_size.restype = ctypes.c_int
        L.glop_batch_workspace_size.argtypes = [vp, u64, u32, ctypes.POINTER(u64)]
        L.glop_scan.restype = ctypes.c_int
        L.glop_scan.argtypes = [vp, vp, u64, vp, u64, vp, vp, u64, vp]
        L.glop_scan_batch.restype = ctypes.c_int
        L.glop_scan_batch.argtypes = [vp, vp, u64, vp, u32, vp, u64, vp, vp, u64, vp]
        L.glop_scan_batch_multi.restype = ctypes.c_int
        L.glop_scan_batch_multi.argtypes = [vp, u32, vp, vp, u64, vp, u32, vp, u64, vp, vp, u64, vp]
        L.glop_batch_multi_kind.restype = ctypes.c_int
        L.glop_batch_multi_kind.argtypes = [vp, ctypes.POINTER(u32)]
        L.glop_scan_status.restype = ctypes.c_int
        L.glop_scan_status.argtypes = [vp, vp, ctypes.POINTER(u64)]
        for name, args in (("glop_server_create", [vp, u32, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]),
                           ("glop_server_submit", [vp, u64, u32, vp, u64]),
                           ("glop_server_poll", [vp, ctypes.POINTER(ServerResult), u32, ctypes.POINTER(u32), u32]),
                           ("glop_server_release", [vp, u64]),
                           ("glop_server_stats_get", [vp, ctypes.POINTER(ServerStats)]),
                           ("glop_server_destroy", [vp])):
            getattr(L, name).restype = ctypes.c_int
            getattr(L, name).argtypes = args
        L.glop_scan_host_staging_size.restype = ctypes.c_int
        L.glop_scan_host_staging_size.argtypes = [vp, u64, u64, ctypes.POINTER(u64)]
        L.glop_scan_host.restype = ctypes.c_int
        L.glop_scan_host.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(u64), vp, u64, vp]
        L.glop_plan_create.restype = ctypes.c_int
        L.glop_plan_create.argtypes = [vp, vp, u64, vp, u32, vp, u64, vp, vp, u64, vp, ctypes.POINTER(vp)]
        L.glop_plan_launch.restype = ctypes.c_int
        L.glop_plan_launch.argtypes = [vp, vp]
        L.glop_plan_destroy.restype = ctypes.c_int
        L.glop_plan_destroy.argtypes = [vp]
        L.glop_tune.restype = ctypes.c_int
        L.glop_tune.argtypes = [vp, vp, u32, u32, vp, u64, vp, u32, u32, ctypes.POINTER(glop_tune_point), u32,
                                ctypes.POINTER(u32), ctypes.POINTER(glop_compile_opts), vp]
        L.glop_scan_noalloc.restype = ctypes.c_int
        L.glop_scan_noalloc.argtypes = [vp, vp, u64, vp, u64, vp, vp]
        L.glop_batch_split.restype = ctypes.c_int
        L.glop_batch_split.argtypes = [vp, vp, u64, ctypes.c_uint32, vp, vp, vp]
        for name, args in (("glop_ingest_create", [vp, u64, u64, ctypes.c_uint32, ctypes.POINTER(vp)]),
                           ("glop_ingest_feed", [vp, vp, u64, ctypes.POINTER(IngestResult)]),
                           ("glop_ingest_flush", [vp, ctypes.POINTER(IngestResult), ctypes.c_uint32,
                                                  ctypes.POINTER(ctypes.c_uint32)]),
                           ("glop_ingest_reset", [vp]),
                           ("glop_ingest_info", [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
                           ("glop_ingest_destroy", [vp])):
            getattr(L, name).restype = ctypes.c_int
            getattr(L, name).argtypes = args
        L.glop_scan_words.restype = ctypes.c_int
        L.glop_scan_words.argtypes = [vp, vp, vp]
        L.glop_scan_host_plan.restype = ctypes.c_int
        L.glop_scan_host_plan.argtypes = [u64, vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
        L.glop_count_workspace_size.restype = ctypes.c_int
        L.glop_count_workspace_size.argtypes = [vp, u64, ctypes.POINTER(u64)]
        L.glop_scan_count.restype = ctypes.c_int
        L.glop_scan_count.argtypes = [vp, vp, u64, vp, vp, vp, u64, vp]
        L.glop_destroy.restype = ctypes.c_int
        L.glop_destroy.argtypes = [vp]
        L.glop_status_str.restype = ctypes.c_char_p
        L.glop_status_str.argtypes = [ctypes.c_int]
        _lib = L
        return L


def _check(rc: int, what: str):
    if rc != OK:
        raise GlopError(rc, what)


def _torch():
    import torch
    return torch


def _pattern_csr(patterns):
    if isinstance(patterns, tuple) and len(patterns) == 2:
        return (np.ascontiguousarray(patterns[0], dtype=np.uint8), np.ascontiguousarray(patterns[1], dtype=np.uint64))
    if hasattr(patterns, "buf") and hasattr(patterns, "offs"):
        return (np.ascontiguousarray(patterns.buf, dtype=np.uint8), np.ascontiguousarray(patterns.offs, dtype=np.uint64))
    pats = [bytes(p) for p in patterns]
    offs = np.zeros(len(pats) + 1, dtype=np.uint64)
    if pats:
        offs[1:] = np.cumsum([len(p) for p in pats])
    buf = np.frombuffer(b"".join(pats), dtype=np.uint8).copy() if pats else np.zeros(1, np.uint8)
    return buf, offs


def _stream_handle(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Automaton:
    """A compiled pattern set resident on the current CUDA device.

    ``patterns``: a list of bytes, or (uint8 buffer, uint64 offsets[n+1]).
    ``prefix_len``: 0 for exact patterns; K > 0 cuts every pattern to K bytes
    (the paper's prefix matching uses K = 8).
    """

    def __init__(self, patterns, prefix_len: int = 0, smem_budget: int = 0, gram_len: int = 0,
                 filter_bits_log2: int = 0, options: dict | None = None, chunk_subtiles: int = 0):
        L = lib()
        buf, offs = _pattern_csr(patterns)
        if buf.size == 0:
            buf = np.zeros(1, np.uint8)
        if options:
            prefix_len = options.get("prefix_len", prefix_len)
            smem_budget = options.get("smem_budget_bytes", smem_budget)
            gram_len = options.get("gram_len", gram_len)
            filter_bits_log2 = options.get("filter_bits_log2", filter_bits_log2)
            chunk_subtiles = options.get("chunk_subtiles", chunk_subtiles)
        opts = glop_compile_opts(prefix_len, smem_budget, 0, gram_len, filter_bits_log2, chunk_subtiles)
        h = ctypes.c_void_p()
        _check(L.glop_compile(buf.ctypes.data, offs.ctypes.data, len(offs) - 1, ctypes.byref(opts),
                              ctypes.byref(h)), "glop_compile")
        self._h = h
        self.n_patterns = len(offs) - 1
        self._ws = {}

    # -- properties
    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise GlopError(EINVAL, "automaton destroyed")
        return self._h

    @property
    def info(self) -> dict:
        inf = glop_info()
        _check(lib().glop_info_get(self.handle, ctypes.byref(inf)), "glop_info_get")
        return {k: getattr(inf, k) for k, _ in glop_info._fields_}

    @property
    def max_pattern_len(self) -> int:
        return int(lib().glop_max_pattern_len(self.handle))

    def workspace_bytes(self, text_len: int, n_segments: int | None = None) -> int:
        v = ctypes.c_uint64()
        if n_segments is None:
            _check(lib().glop_scan_workspace_size(self.handle, text_len, ctypes.byref(v)), "workspace size")
        else:
            _check(lib().glop_batch_workspace_size(self.handle, text_len, n_segments, ctypes.byref(v)), "ws size")
        return int(v.value)

    def workspace(self, text_len: int, device, n_segments: int | None = None):
        """A cached device workspace large enough for text_len bytes."""
        torch = _torch()
        need = self.workspace_bytes(text_len, n_segments)
        key = (str(device), n_segments is not None)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=device)
            self._ws[key] = ws
        return ws

    # -- scans
    def scan_into(self, text, matches, count, workspace=None, stream=None) -> None:
        """Queue a scan of ``text`` (uint8 CUDA tensor) writing ``matches`` ((cap, 2) int32 CUDA
        tensor) and ``count`` (int64 CUDA tensor of one element).  Asynchronous."""
        n = text.numel()
        ws = workspace if workspace is not None else self.workspace(n, text.device)
        cap = matches.shape[0] if matches is not None else 0
        _check(lib().glop_scan(self.handle, text.data_ptr() if n else None, n,
                               matches.data_ptr() if cap else None, cap, count.data_ptr(),
                               ws.data_ptr(), ws.numel(), _stream_handle(stream)), "glop_scan")

    def scan(self, text, capacity: int | None = None, stream=None):
        """All matches of a uint8 CUDA tensor: ((M, 2) int32 tensor of (offset, pattern_id), M).

        The capacity is grown and the scan repeated when the first guess is too small."""
        torch = _torch()
        n = text.numel()
        cap = capacity if capacity is not None else max(1024, n // 4)
        count = torch.zeros(1, dtype=torch.int64, device=text.device)
        while True:
            m = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=text.device)
            self.scan_into(text, m, count, stream=stream)
            st = self.status(text.device, stream=stream)
            total = int(count.item())
            if total <= cap:
                if st not in (OK,):
                    raise GlopError(st, "scan")
                return m[:total], total
            if capacity is not None:
                raise GlopError(EOVERFLOW, "%d matches > capacity %d" % (total, cap))
            cap = total

    def status(self, device, stream=None, batch: bool = False) -> int:
        ws = self._ws.get((str(device), batch))
        if ws is None:
            return OK
        cnt = ctypes.c_uint64()
        return int(lib().glop_scan_status(ws.data_ptr(), _stream_handle(stream), ctypes.byref(cnt)))

    def scan_batch_into(self, text, seg_offsets, matches, count, workspace=None, stream=None) -> None:
        """Queue a batch scan: ``seg_offsets`` int64 CUDA tensor of n+1 offsets; ``matches`` (cap, 3) int32."""
        n = text.numel()
        nseg = seg_offsets.numel() - 1
        ws = workspace if workspace is not None else self.workspace(n, text.device, nseg)
        cap = matches.shape[0] if matches is not None else 0
        _check(lib().glop_scan_batch(self.handle, text.data_ptr() if n else None, n, seg_offsets.data_ptr(), nseg,
                                     matches.data_ptr() if cap else None, cap, count.data_ptr(), ws.data_ptr(),
                                     ws.numel(), _stream_handle(stream)), "glop_scan_batch")

    def scan_batch(self, text, seg_offsets, capacity: int | None = None, stream=None):
        """All matches per segment: ((M, 3) int32 tensor of (segment, offset, pattern_id), M)."""
        torch = _torch()
        n = text.numel()
        cap = capacity if capacity is not None else max(1024, n // 4)
        count = torch.zeros(1, dtype=torch.int64, device=text.device)
        while True:
            m = torch.empty((max(cap, 1), 3), dtype=torch.int32, device=text.device)
            self.scan_batch_into(text, seg_offsets, m, count, stream=stream)
            st = self.status(text.device, stream=stream, batch=True)
            total = int(count.item())
            if st == EINVAL:
                raise GlopError(EINVAL, "malformed segment offsets")
            if total <= cap:
                if st != OK:
                    raise GlopError(st, "scan_batch")
                return m[:total], total
            if capacity is not None:
                raise GlopError(EOVERFLOW, "%d matches > capacity %d" % (total, cap))
            cap = total

    def count_workspace(self, device):
        """A cached device workspace for count_into on this handle."""
        torch = _torch()
        need = ctypes.c_uint64()
        _check(lib().glop_count_workspace_size(self.handle, 0, ctypes.byref(need)), "count workspace size")
        ws = getattr(self, "_count_ws", None)
        if ws is None or ws.numel() < need.value or ws.device != torch.device(device):
            ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=device)
            self._count_ws = ws
        return ws

    def count_into(self, text, hist, total, workspace=None, stream=None) -> None:
        """Queue a count-only scan: ``hist`` (int64 CUDA tensor of n_patterns) gets each pattern's number of
        occurrences in ``text``, ``total`` (int64, one element) their sum.  Asynchronous."""
        torch = _torch()
        ws = workspace if workspace is not None else self.count_workspace(text.device)
        st = stream if stream is not None else torch.cuda.current_stream(text.device)
        _check(lib().glop_scan_count(self.handle, text.data_ptr(), text.numel(), hist.data_ptr(), total.data_ptr(),
                                     ws.data_ptr(), ws.numel(), st.cuda_stream), "glop_scan_count")

    def count(self, text, stream=None):
        """Per-pattern occurrence counts of ``text`` (uint8 CUDA tensor): (int64 tensor of n_patterns, total)."""
        torch = _torch()
        n = max(self.info["n_patterns"], 1)
        hist = torch.empty(n, dtype=torch.int64, device=text.device)
        total = torch.empty(1, dtype=torch.int64, device=text.device)
        ws = self.count_workspace(text.device)
        self.count_into(text, hist, total, workspace=ws, stream=stream)
        st = lib().glop_scan_status(ws.data_ptr(), (stream or torch.cuda.current_stream(text.device)).cuda_stream,
                                    None)
        if st != OK:
            raise GlopError(st, "glop_scan_count")
        return hist[:self.info["n_patterns"]], int(total.item())

    def scan_host(self, text: np.ndarray, capacity: int, staging=None, stream=None):
        """End-to-end scan of a HOST uint8 array (pinned is fastest): copies in, scans, copies back.
        Returns ((M, 2) uint32 numpy array, total count)."""
        torch = _torch()
        t = np.ascontiguousarray(text, dtype=np.uint8).reshape(-1)
        need = ctypes.c_uint64()
        _check(lib().glop_scan_host_staging_size(self.handle, t.size, capacity, ctypes.byref(need)), "staging")
        if staging is None:
            staging = torch.empty(int(need.value), dtype=torch.uint8, device="cuda")
        out = np.empty((max(capacity, 1), 2), dtype=np.uint32)
        cnt = ctypes.c_uint64()
        rc = lib().glop_scan_host(self.handle, t.ctypes.data if t.size else None, t.size, out.ctypes.data, capacity,
                                  ctypes.byref(cnt), staging.data_ptr(), staging.numel(), _stream_handle(stream))
        if rc not in (OK, EOVERFLOW):
            raise GlopError(rc, "glop_scan_host")
        total = int(cnt.value)
        return out[:min(total, capacity)], total

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().glop_destroy(self._h)
            self._h = None
        self._ws = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_plan(length: int) -> list:
    """Piece boundaries glop_scan_host uses for a ``length``-byte text: [0, ..., length]."""
    n = ctypes.c_uint32()
    _check(lib().glop_scan_host_plan(length, None, 0, ctypes.byref(n)), "glop_scan_host_plan")
    b = (ctypes.c_uint64 * (n.value + 1))()
    _check(lib().glop_scan_host_plan(length, b, n.value + 1, ctypes.byref(n)), "glop_scan_host_plan")
    return [int(x) for x in b]


def batch_split(matches, count, n_segments: int, pairs, seg_first, stream=None) -> None:
    """Queue glop_batch_split: ``matches`` ((cap, 3) int32 CUDA tensor from a batch scan), ``count`` (its
    int64 count) -> ``pairs`` ((cap, 2) int32) and ``seg_first`` (int64, n_segments + 1).  Asynchronous."""
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream(matches.device)
    cap = matches.shape[0]
    if pairs.shape[0] < cap or seg_first.numel() < n_segments + 1:
        raise GlopError(EINVAL, "batch_split: output too small")
    _check(lib().glop_batch_split(matches.data_ptr(), count.data_ptr(), cap, n_segments, pairs.data_ptr(),
                                  seg_first.data_ptr(), st.cuda_stream), "glop_batch_split")


class Plan:
    """A scan captured into a CUDA graph for fixed device buffers; ``launch()`` replays it with one graph launch.

    ``seg_offsets`` None: single-buffer scan, ``matches`` (cap, 2) int32; else a batch over segments, ``matches``
    (cap, 3) int32.  All tensors must outlive the plan.  ``stream`` must be a non-default torch stream."""

    def __init__(self, automaton: Automaton, text, matches, count, seg_offsets=None, stream=None):
        torch = _torch()
        self._keep = (automaton, text, matches, count, seg_offsets)
        n = text.numel()
        nseg = None if seg_offsets is None else seg_offsets.numel() - 1
        self.workspace = torch.empty(automaton.workspace_bytes(n, nseg), dtype=torch.uint8, device=text.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=text.device)
        h = ctypes.c_void_p()
        _check(lib().glop_plan_create(automaton.handle, text.data_ptr() if n else None, n,
                                      None if seg_offsets is None else seg_offsets.data_ptr(), nseg or 0,
                                      matches.data_ptr(), matches.shape[0], count.data_ptr(),
                                      self.workspace.data_ptr(), self.workspace.numel(), self.stream.cuda_stream,
                                      ctypes.byref(h)), "glop_plan_create")
        self._h = h

    def launch(self, stream=None) -> None:
        s = stream if stream is not None else self.stream
        _check(lib().glop_plan_launch(self._h, s.cuda_stream), "glop_plan_launch")

    def status(self, stream=None) -> int:
        s = stream if stream is not None else self.stream
        cnt = ctypes.c_uint64()
        return int(lib().glop_scan_status(self.workspace.data_ptr(), s.cuda_stream, ctypes.byref(cnt)))

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().glop_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_multi_kind(a: "Automaton") -> int:
    """The kernel kind of an automaton: automata of equal kinds can share one scan_batch_multi launch."""
    k = ctypes.c_uint32()
    _check(lib().glop_batch_multi_kind(a.handle, ctypes.byref(k)), "glop_batch_multi_kind")
    return int(k.value)


def scan_batch_multi_into(automata, group_start, text, seg_offsets, matches, count, workspace, stream=None) -> None:
    """Queue one batch scan over segments of several automata (glop_scan_batch_multi): group g is the text
    [group_start[g], group_start[g + 1]) (host ints, multiples of 1024, each the start of a segment),
    scanned with automata[g]; writes (segment, offset, pattern_id) rows to ``matches`` and the total to
    ``count``.  Asynchronous."""
    n = len(automata)
    hs = (ctypes.c_void_p * n)(*[a.handle.value for a in automata])
    gs = np.ascontiguousarray(group_start, dtype=np.uint64)
    cap = matches.shape[0] if matches is not None else 0
    nseg = seg_offsets.numel() - 1
    _check(lib().glop_scan_batch_multi(hs, n, gs.ctypes.data, text.data_ptr() if text.numel() else None,
                                       text.numel(), seg_offsets.data_ptr(), nseg,
                                       matches.data_ptr() if cap else None, cap, count.data_ptr(),
                                       workspace.data_ptr(), workspace.numel(), _stream_handle(stream)),
           "glop_scan_batch_multi")


def _opts_dict(o: glop_compile_opts) -> dict:
    return {k: int(getattr(o, k)) for k, _ in glop_compile_opts._fields_ if k != "flags"}


def tune(patterns, sample, seg_offsets=None, prefix_len: int = 0, repeats: int = 5, cache_path: str | None = None,
         stream=None) -> dict:
    """Autotune compile options on a sample (uint8 CUDA tensor; a batch when ``seg_offsets`` is given).

    Returns ``{"best": options, "points": [...], "cached": bool}``.  With ``cache_path`` (default: the
    GLOP_TUNE_CACHE environment variable) results are kept in a JSON file keyed by the pattern set, the
    prefix length, the sample's size/kind and the device name."""
    import hashlib
    import json
    torch = _torch()
    buf, offs = _pattern_csr(patterns)
    cache_path = cache_path or os.environ.get("GLOP_TUNE_CACHE")
    key = "|".join([hashlib.sha256(buf.tobytes() + offs.tobytes()).hexdigest()[:32], str(prefix_len),
                    "batch" if seg_offsets is not None else "single", str(sample.numel()),
                    torch.cuda.get_device_name(sample.device)])
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
        if key in cache:
            return dict(cache[key], cached=True)
    if buf.size == 0:
        buf = np.zeros(1, np.uint8)
    maxp = 64
    pts = (glop_tune_point * maxp)()
    npts = ctypes.c_uint32()
    best = glop_compile_opts()
    nseg = 0 if seg_offsets is None else seg_offsets.numel() - 1
    _check(lib().glop_tune(buf.ctypes.data, offs.ctypes.data, len(offs) - 1, prefix_len, sample.data_ptr(),
                           sample.numel(), None if seg_offsets is None else seg_offsets.data_ptr(), nseg, repeats,
                           pts, maxp, ctypes.byref(npts), ctypes.byref(best), _stream_handle(stream)), "glop_tune")
    res = {"best": _opts_dict(best),
           "points": [dict(_opts_dict(pts[i].opts), gbps=round(pts[i].gbps, 2)) for i in range(min(npts.value, maxp))]}
    if cache_path:
        cache[key] = res
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(res, cached=False)

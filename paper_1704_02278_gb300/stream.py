"""Streaming ingestion: a log stream scanned chunk by chunk as it arrives.

The paper streams the next batch of logs to the GPU while the current one is
scanned (Sec. 6) and names real-time operation as the goal (Sec. 8); Sec. 4
fixes what chunked scanning must carry over: an overlap of the longest
pattern - 1 bytes.  Here:

* every scan covers the carried tail of the previous chunk (``halo`` =
  longest pattern - 1 bytes, copied device to device) plus the new chunk;
* a scan owns the match starts in ``[buffer start, buffer end - halo)``: a
  match starting in the last ``halo`` bytes may run past the bytes seen so
  far, so it is left to the next scan, whose buffer starts exactly there;
  ``flush`` owns everything up to the end of the stream.  The owned matches
  are a prefix of the scan's sorted output;
* ``depth + 1`` slots, each with its own CUDA stream, device buffers and
  pinned result rows, rotate: one chunk's host-to-device copy and scan run
  while the previous chunk's matches are copied back and the results of the
  one before are handed out, in stream order.

The engine is native (``glop_ingest_*`` in the C ABI) and this module wraps
it; ``owned_end`` states the ownership rule the engine applies.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Automaton, GlopError, IngestResult, OK, lib


def owned_end(buf_start: int, buf_end: int, halo: int, final: bool) -> int:
    """End (exclusive) of the match starts a scan of stream bytes [buf_start, buf_end) owns."""
    return buf_end if final else max(buf_start, buf_end - halo)


class StreamResult:
    """The owned matches of one scan: ``matches`` is a (k, 2) uint32 view (offset relative to ``base``,
    pattern_id), sorted, of the scanning slot's pinned buffer -- valid until that slot's next copy-back is
    queued, in the second ``feed`` call after the one that returned it; ``absolute()`` copies it out with
    uint64 stream offsets."""

    def __init__(self, base: int, matches: np.ndarray):
        self.base = base
        self.matches = matches

    def __len__(self) -> int:
        return len(self.matches)

    def absolute(self) -> np.ndarray:
        out = self.matches.astype(np.uint64)
        out[:, 0] += np.uint64(self.base)
        return out


_NONE = np.zeros((0, 2), np.uint32)


class _Same:
    """No device change (a context manager that does nothing)."""

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


class StreamScanner:
    """Scan a byte stream fed in chunks of at most ``chunk_bytes`` (pinned host memory is fastest).

    ``feed(chunk)`` queues the chunk and returns the results of the chunk fed ``depth`` calls before it (an
    empty result while fewer were fed); ``flush()`` returns the rest, as a list.  Each result is a
    StreamResult; in order, their matches are exactly the matches of the whole stream.  A chunk must stay
    unchanged until the next ``feed`` (or ``flush``) returns; the scanner keeps a reference to it."""

    def __init__(self, patterns, chunk_bytes: int = 16 << 20, out_rows: int | None = None, prefix_len: int = 0,
                 device=None, depth: int = 2):
        # the engine works on the device current at creation; `device` makes it current for every call
        self._ctx = None
        if device is not None:
            import torch
            self._ctx = torch.cuda.device(device)
        self.chunk_bytes = chunk_bytes
        self.depth = int(depth)
        self.lib = lib()
        h = ctypes.c_void_p()
        with self._ctx or _Same():
            self.a = patterns if isinstance(patterns, Automaton) else Automaton(patterns, prefix_len=prefix_len)
            rc = self.lib.glop_ingest_create(self.a.handle, chunk_bytes, out_rows or 0, self.depth, ctypes.byref(h))
        self.halo = max(int(self.a.info["max_pattern_len"]) - 1, 0)
        if rc != OK:
            raise GlopError(rc, "glop_ingest_create")
        self._h = h
        self._res = IngestResult()
        self._hold = []  # the chunks whose uploads may still be running

    @property
    def stats(self) -> dict:
        chunks, rescans = ctypes.c_uint64(), ctypes.c_uint64()
        self.lib.glop_ingest_info(self._h, ctypes.byref(chunks), ctypes.byref(rescans))
        return {"chunks": chunks.value, "rescans": rescans.value}

    @staticmethod
    def _result(r: IngestResult) -> StreamResult:
        n = int(r.count)
        if n == 0:
            return StreamResult(int(r.base), _NONE)
        rows = np.frombuffer((ctypes.c_uint32 * (2 * n)).from_address(r.matches), dtype=np.uint32)
        return StreamResult(int(r.base), rows.reshape(n, 2))

    def feed(self, chunk) -> StreamResult:
        """Queue the next chunk (uint8 numpy array or CPU tensor, at most chunk_bytes); return the owned
        matches of the chunk fed ``depth`` calls before."""
        if isinstance(chunk, np.ndarray):
            buf = np.ascontiguousarray(chunk, dtype=np.uint8).reshape(-1)
            ptr, n = buf.ctypes.data, buf.size
        else:  # a CPU tensor
            buf = chunk if chunk.is_contiguous() else chunk.contiguous()
            ptr, n = buf.data_ptr(), buf.numel()
        if n > self.chunk_bytes:
            raise GlopError(1, "chunk of %d bytes > chunk_bytes %d" % (n, self.chunk_bytes))
        with self._ctx or _Same():
            rc = self.lib.glop_ingest_feed(self._h, ptr if n else None, n, ctypes.byref(self._res))
        if rc != OK:
            raise GlopError(rc, "glop_ingest_feed")
        self._hold = [self._hold[-1], buf] if self._hold else [buf]
        return self._result(self._res)

    def flush(self) -> list:
        """Finish the stream: the results of every chunk not yet returned, in order; the last scan owns every
        remaining start."""
        res = (IngestResult * max(self.depth, 1))()
        got = ctypes.c_uint32()
        with self._ctx or _Same():
            rc = self.lib.glop_ingest_flush(self._h, res, len(res), ctypes.byref(got))
        if rc != OK:
            raise GlopError(rc, "glop_ingest_flush")
        self._hold = []
        return [self._result(res[i]) for i in range(got.value)]

    def reset(self):
        """Start a new stream (the previous one must have been flushed)."""
        rc = self.lib.glop_ingest_reset(self._h)
        if rc != OK:
            raise GlopError(rc, "glop_ingest_reset (flush first)")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.glop_ingest_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

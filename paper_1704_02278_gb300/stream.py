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
  pinned result buffer, rotate: one chunk's host-to-device copy and scan run
  while the previous chunk's matches are copied back and the host hands out
  the results of the one before, in stream order.

All matching runs in the library's kernels (``glop_scan``); this module
moves bytes and keeps the books.
"""
from __future__ import annotations

import bisect

import numpy as np

from . import Automaton, GlopError, OK, lib


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


_EMPTY = StreamResult(0, np.zeros((0, 2), np.uint32))


class _Slot:
    def __init__(self, torch, device, cap_bytes: int, out_rows: int, ws_bytes: int):
        self.stream = torch.cuda.Stream(device=device)
        self.text = torch.empty(cap_bytes, dtype=torch.uint8, device=device)
        self.out = torch.empty((out_rows, 2), dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
        self.count_host = torch.empty(1, dtype=torch.int64, pin_memory=True)
        self.out_host = torch.empty((out_rows, 2), dtype=torch.int32, pin_memory=True)
        self.last_len = 0
        self.uploaded = torch.cuda.Event()  # the chunk's bytes are on the device
        self.done = torch.cuda.Event()      # the scan and its match count's copy-back finished
        self.copied = torch.cuda.Event()    # the scan's matches are in out_host


class _Pending:
    """A queued scan whose results have not been returned: stream bytes [b0, b1) in ``slot``."""

    def __init__(self, slot, b0: int, b1: int):
        self.slot, self.b0, self.b1 = slot, b0, b1
        self.n = -1  # match count, once the scan is over and its copy-back is queued


class StreamScanner:
    """Scan a byte stream fed in chunks of at most ``chunk_bytes`` (pinned host memory is fastest).

    ``feed(chunk)`` queues the chunk and returns the results of the chunk fed ``depth`` calls before it (an
    empty result while fewer were fed); ``flush()`` returns the rest, as a list.  Each result is a
    StreamResult; in order, their matches are exactly the matches of the whole stream.  ``depth + 1`` slots
    rotate: with ``depth`` = 2, one chunk uploads and scans while the previous chunk's matches copy back and
    the one before is handed out, so the host's own work overlaps the device's."""

    def __init__(self, patterns, chunk_bytes: int = 16 << 20, out_rows: int | None = None, prefix_len: int = 0,
                 device=None, depth: int = 2):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.a = patterns if isinstance(patterns, Automaton) else Automaton(patterns, prefix_len=prefix_len)
        self.halo = max(int(self.a.info["max_pattern_len"]) - 1, 0)
        self.chunk_bytes = chunk_bytes
        self.depth = max(1, int(depth))
        cap = chunk_bytes + self.halo
        rows = out_rows if out_rows is not None else max(1 << 16, cap // 4)
        ws = self.a.workspace_bytes(cap)
        self.slots = [_Slot(torch, self.device, cap, rows, ws) for _ in range(self.depth + 1)]
        self.lib = lib()
        self.stats = {"chunks": 0, "rescans": 0}
        self.reset()

    def reset(self):
        """Start a new stream (the previous one must have been flushed)."""
        self.pos = 0          # stream bytes fed so far
        self.buf_start = 0    # stream offset of the next scan's buffer start
        self.k = 0            # chunks fed
        self.pending = []     # queued scans whose results are not yet returned, oldest first
        self.tail_slot = None  # slot whose device buffer ends with the bytes to carry
        self.tail_len = 0

    def _start_copy(self, e: _Pending):
        """Wait for the scan of e, then queue the copy-back of exactly its matches."""
        torch = self.torch
        s = e.slot
        s.done.synchronize()
        n = int(s.count_host.item())
        if n > s.out.shape[0]:
            # more matches than the output holds: scan the same buffer again into a larger one
            self.stats["rescans"] += 1
            s.out = torch.empty((n, 2), dtype=torch.int32, device=self.device)
            self._scan(s, e.b1 - e.b0)
            s.done.synchronize()
        if s.out_host.shape[0] < n:
            s.out_host = torch.empty((n, 2), dtype=torch.int32, pin_memory=True)
        if n:
            with torch.cuda.stream(s.stream):
                s.out_host[:n].copy_(s.out[:n], non_blocking=True)
        s.copied.record(s.stream)
        e.n = n

    def _finish(self, e: _Pending, final: bool) -> StreamResult:
        """Wait for the copy-back of e and return its owned matches."""
        if e.n < 0:
            self._start_copy(e)
        s = e.slot
        s.copied.synchronize()
        n = e.n
        m = s.out_host[:n].numpy().view(np.uint32)
        end = owned_end(e.b0, e.b1, self.halo, final) - e.b0
        # first row at or past the owned end (binary search on the strided column, no copy of it)
        col = m[:, 0]
        keep = bisect.bisect_left(range(n), end, key=lambda i: int(col[i]))
        return StreamResult(e.b0, m[:keep])

    def _scan(self, s, nbytes: int):
        torch = self.torch
        rc = self.lib.glop_scan(self.a.handle, s.text.data_ptr(), nbytes, s.out.data_ptr(), s.out.shape[0],
                                s.count.data_ptr(), s.ws.data_ptr(), s.ws.numel(), s.stream.cuda_stream)
        if rc != OK:
            raise GlopError(rc, "glop_scan")
        with torch.cuda.stream(s.stream):
            s.count_host.copy_(s.count, non_blocking=True)
        s.done.record(s.stream)

    def feed(self, chunk) -> StreamResult:
        """Queue the next chunk (uint8 numpy array or CPU tensor, at most chunk_bytes); return the owned
        matches of the chunk fed ``depth`` calls before."""
        torch = self.torch
        t = chunk if isinstance(chunk, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(chunk, np.uint8))
        n = t.numel()
        if n > self.chunk_bytes:
            raise GlopError(1, "chunk of %d bytes > chunk_bytes %d" % (n, self.chunk_bytes))
        nslot = len(self.slots)
        s = self.slots[self.k % nslot]
        prev = self.slots[(self.k - 1) % nslot]
        h = self.tail_len
        with torch.cuda.stream(s.stream):
            if self.k:
                # every earlier upload, and the tail copy that read this slot's old bytes, come first (each
                # upload waits for the one before it)
                s.stream.wait_event(prev.uploaded)
            if h:
                # the carried bytes: the end of the previous buffer
                p = self.tail_slot
                s.text[:h].copy_(p.text[p.last_len - h:p.last_len], non_blocking=True)
            s.text[h:h + n].copy_(t, non_blocking=True)
        s.uploaded.record(s.stream)
        s.last_len = h + n
        b0 = self.buf_start
        b1 = b0 + h + n
        # queue this chunk's scan, then, while it runs, queue the previous scan's copy-back and hand out the
        # results of the chunk fed `depth` calls ago
        self._scan(s, h + n)
        self.pending.append(_Pending(s, b0, b1))
        if len(self.pending) >= 2 and self.pending[-2].n < 0:
            self._start_copy(self.pending[-2])
        out = self._finish(self.pending.pop(0), final=False) if len(self.pending) > self.depth else _EMPTY
        # next buffer starts where this scan's ownership ends
        nxt = owned_end(b0, b1, self.halo, False)
        self.tail_len = b1 - nxt
        self.tail_slot = s
        self.buf_start = nxt
        self.pos += n
        self.k += 1
        self.stats["chunks"] += 1
        return out

    def flush(self) -> list:
        """Finish the stream: the results of every chunk not yet returned, in order; the last scan owns every
        remaining start."""
        for e in self.pending:
            if e.n < 0:
                self._start_copy(e)
        out = []
        while self.pending:
            e = self.pending.pop(0)
            out.append(self._finish(e, final=not self.pending))
        return out

    def close(self):
        for s in self.slots:
            s.done.synchronize()
            s.copied.synchronize()

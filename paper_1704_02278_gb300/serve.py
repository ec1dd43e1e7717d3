"""Continuous-batching scan server over device-resident automata.

The paper's use case (Sec. 1) pushes syslog traces and rules to a GPU server
that answers with the number and locations of suspect events; its library
streams the next batch of logs while a kernel runs (Sec. 6) and names
real-time operation as future work (Sec. 8).  This module is that serving
layer: several compiled pattern sets stay resident on the device, requests
(payload bytes + the set to scan with) arrive over time, and the loop

* admits a request when its payload, scratch and estimated output fit in a
  device-memory budget (an arena of one allocation, first-fit),
* batches the admitted requests into a single launch (one segment per
  request) while earlier batches are still on the GPU: requests for several
  resident sets of one kernel kind share a ``glop_scan_batch_multi`` launch,
  one group of segments per set, each group scanned with its own automaton --
  up to ``max_inflight`` batches overlap, each on its own stream, so copies
  of one batch run under the scan of another,
* sends a request of at least ``big_bytes`` to a lane of its own: a worker
  thread that scans it end to end through ``glop_scan_host`` (uploads, scans
  and copy-backs of its pieces overlapped) into a pinned result buffer sized
  up front, so a large request neither waits for a batch nor holds the
  batches of small requests behind it,
* returns each request's matches as (offset, pattern_id) pairs and its
  latency from arrival to results on the host.

``PlainServer`` is the baseline: one request at a time, in arrival order,
through the end-to-end ``glop_scan_host`` call.

The scan arithmetic is the library's (``libglop.so``); this module only
schedules, moves bytes and keeps books.
"""
from __future__ import annotations

import bisect
import ctypes
import dataclasses
import time

import numpy as np

from . import Automaton, GlopError, lib, EOVERFLOW, OK, batch_multi_kind
from . import ServerOpts as _ServerOpts, ServerResult as _ServerResult, ServerStats as _ServerStats

MAX_GROUPS = 8   # pattern sets in one batch launch (glop_scan_batch_multi)
GROUP_ALIGN = 1024  # every set's group of segments starts on this byte boundary


@dataclasses.dataclass
class Request:
    rid: int
    set_index: int
    payload: object          # pinned CPU uint8 torch tensor (a view is fine)
    arrival: float           # seconds from the start of the run
    # filled in by the server
    done: float = -1.0
    count: int = -1
    matches: np.ndarray | None = None  # (count, 2) uint32 (offset, pattern_id) when kept


class DeviceArena:
    """First-fit allocator over one device allocation of ``budget`` bytes (the HBM budget)."""

    ALIGN = 256

    def __init__(self, budget: int, device):
        import torch
        self.buf = torch.empty(budget, dtype=torch.uint8, device=device)
        self.base = self.buf.data_ptr()
        self.size = budget
        self.free = [(0, budget)]  # sorted (offset, length)

    def alloc(self, n: int):
        n = (max(n, 1) + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                return off, n
        return None

    def release(self, off: int, n: int):
        bisect.insort(self.free, (off, n))
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    def view(self, off: int, n: int):
        return self.buf[off:off + n]

    @property
    def largest_free(self) -> int:
        return max((ln for _, ln in self.free), default=0)


class _Slot:
    """Per-stream resources reused by every batch the stream carries (nothing is allocated per batch)."""

    def __init__(self, torch, device, max_requests: int, out_rows: int):
        self.stream = torch.cuda.Stream(device=device)
        # segments: one per request, plus one padding segment per group of a multi-set batch
        self.seg_host = torch.empty(max_requests + 1 + MAX_GROUPS, dtype=torch.int64, pin_memory=True)
        self.first_host = torch.empty(max_requests + 1 + MAX_GROUPS, dtype=torch.int64, pin_memory=True)
        self.count_host = torch.empty(1, dtype=torch.int64, pin_memory=True)
        self.out_host = torch.empty((out_rows, 2), dtype=torch.int32, pin_memory=True)
        self.ev = torch.cuda.Event()
        self.extra = None  # device outputs of a rescan

    def host_out(self, torch, n: int, keep: int = 0):
        """The pinned pair buffer with room for n rows (its first keep rows preserved when it grows)."""
        if self.out_host.shape[0] < n:
            old = self.out_host
            self.out_host = torch.empty((max(n, 2 * old.shape[0]), 2), dtype=torch.int32, pin_memory=True)
            if keep:
                self.out_host[:keep].copy_(old[:keep])
        return self.out_host


class _Batch:
    pass


class _BigLane:
    """One worker thread serving large requests in arrival order through the end-to-end glop_scan_host call
    (pieces uploaded, scanned and copied back overlapped) on its own stream, staging and pinned result rows.
    The library call releases the interpreter lock, so the serving loop keeps batching meanwhile."""

    def __init__(self, torch, device, automata, max_bytes: int, out_rows: int, keep: bool):
        import queue
        import threading
        self.torch, self.device, self.automata, self.keep = torch, device, automata, keep
        self.lib = lib()
        self.max_bytes = max_bytes
        self.stream = torch.cuda.Stream(device=device, priority=-1)  # latency first: ahead of batch kernels
        self._size(out_rows)
        self.q = queue.Queue()
        self.completed = 0
        self.rescans = 0
        self.error = None
        self.t0 = 0.0
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def _size(self, rows: int):
        torch = self.torch
        need = ctypes.c_uint64()
        self.lib.glop_scan_host_staging_size(self.automata[0].handle, self.max_bytes, rows, ctypes.byref(need))
        self.staging = torch.empty(int(need.value), dtype=torch.uint8, device=self.device)
        self.out = torch.empty((rows, 2), dtype=torch.int32, pin_memory=True)
        self.rows = rows

    def _run(self):
        torch = self.torch
        cnt = ctypes.c_uint64()
        try:
            dev = self.device.index if self.device.index is not None else torch.cuda.current_device()
            torch.cuda.set_device(dev)
        except Exception as e:  # reported by the serving loop; requests still count as finished
            self.error = e
        while True:
            r = self.q.get()
            if r is None:
                return
            if self.error is not None:
                self.completed += 1
                continue
            try:
                n = r.payload.numel()
                while True:
                    rc = self.lib.glop_scan_host(self.automata[r.set_index].handle, r.payload.data_ptr(), n,
                                                 self.out.data_ptr(), self.rows, ctypes.byref(cnt),
                                                 self.staging.data_ptr(), self.staging.numel(),
                                                 self.stream.cuda_stream)
                    if rc == EOVERFLOW:  # more matches than the rows sized up front: grow once and scan again
                        self.rescans += 1
                        self._size(int(cnt.value) + (1 << 20))
                        continue
                    if rc != OK:
                        raise GlopError(rc, "glop_scan_host")
                    break
                r.count = int(cnt.value)
                if self.keep:
                    r.matches = self.out[:r.count].numpy().view(np.uint32).copy()
                r.done = time.perf_counter() - self.t0
            except Exception as e:  # reported by the serving loop
                self.error = e
            self.completed += 1

    def close(self):
        self.q.put(None)
        self.thread.join()


class BatchServer:
    """Continuous batching of scan requests over resident automata (see module doc).

    Pending requests wait in one FIFO per pattern set.  A batch takes the set
    of the oldest pending request and as many of that set's requests, in
    arrival order, as fit ``max_batch_bytes``, ``max_batch_requests``, the
    pinned result buffer of a stream slot and the largest free block of the
    device arena (the group is halved until it fits).  After the scan,
    ``glop_batch_split`` turns the batch's (segment, offset, pattern_id)
    matches into (offset, pattern_id) pairs and per-request runs, and only
    those come back over the host link: the match count and the runs first
    (with the pairs too when the output bound is small), then exactly the
    pairs that exist.  The output bound comes from a running estimate of
    matches per byte of the set (a decaying maximum); a batch that outgrows
    it is scanned again."""

    EAGER_ROWS = 1 << 16  # output bounds up to this many pairs come back with the count, in one round

    def __init__(self, pattern_sets, hbm_budget: int = 8 << 30, max_inflight: int = 4,
                 max_batch_bytes: int = 256 << 20, max_batch_requests: int = 512, keep_matches: bool = False,
                 out_rows: int | None = None, fast_bytes: int = 1 << 20, big_bytes: int = 8 << 20,
                 max_request_bytes: int = 0, big_out_rows: int | None = None, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.automata = [Automaton(p) for p in pattern_sets]
        self.arena = DeviceArena(hbm_budget, self.device)
        if out_rows is None:  # pinned result pairs per stream slot: 1 per 16 bytes of the largest batch
            out_rows = max(1 << 16, min(max_batch_bytes, hbm_budget) // 16)
        self.slots = [_Slot(torch, self.device, max_batch_requests, out_rows) for _ in range(max_inflight)]
        self.max_inflight = max_inflight
        self.max_batch_bytes = max_batch_bytes
        self.max_batch_requests = max_batch_requests
        self.out_rows = out_rows
        self.keep = keep_matches
        # matches per payload byte per set: a slowly decaying maximum over recent batches (request content
        # varies, and an output bound that is too small costs a second scan)
        self.density = [0.25] * len(self.automata)
        # sets whose automata share a kernel kind can share one launch
        self.kind = [batch_multi_kind(a) for a in self.automata]
        self.lib = lib()
        self.stats = {}
        # idle fast path: a lone request of at most fast_bytes while nothing is in flight goes through one
        # end-to-end glop_scan_host call (copy in, scan, copy back), as a plain loop would
        self.fast_bytes = fast_bytes
        self.fast_cap = max(1 << 16, fast_bytes)
        if fast_bytes:
            need = ctypes.c_uint64()
            self.lib.glop_scan_host_staging_size(self.automata[0].handle, fast_bytes, self.fast_cap,
                                                 ctypes.byref(need))
            self.fast_staging = torch.empty(int(need.value), dtype=torch.uint8, device=self.device)
            self.fast_out = torch.empty((self.fast_cap, 2), dtype=torch.int32, pin_memory=True)
            self.fast_stream = torch.cuda.Stream(device=self.device, priority=-1)
        # the lane for requests of at least big_bytes (0 = none): sized for max_request_bytes, with result rows
        # for two matches per payload byte unless big_out_rows says otherwise
        self.big_bytes = big_bytes if max_request_bytes >= big_bytes > 0 else 0
        self.big = None
        if self.big_bytes:
            rows = big_out_rows if big_out_rows is not None else 2 * max_request_bytes
            self.big = _BigLane(torch, self.device, self.automata, max_request_bytes, max(rows, 1 << 16),
                                keep_matches)

    def close(self):
        """Stop the large-request worker (the server is unusable afterwards)."""
        if self.big is not None:
            self.big.close()
            self.big = None

    # -- one batch -------------------------------------------------------------
    # A batch is a list of groups (set index, requests of that set in arrival order).  Its text holds the
    # groups one after another, each starting on a GROUP_ALIGN boundary (the gap before the next group is a
    # padding segment whose matches nobody reads); one segment per request.
    def _cap(self, groups) -> int:
        return int(sum(self.density[si] * sum(r.payload.numel() for r in rs) for si, rs in groups) * 1.25) + 4096

    @staticmethod
    def _layout(groups):
        """(text bytes, segment ends, group starts, segment of each request in batch order)."""
        ends, gstart, rseg = [], [], []
        pos = 0
        for gi, (si, rs) in enumerate(groups):
            gstart.append(pos)
            for r in rs:
                pos += r.payload.numel()
                ends.append(pos)
                rseg.append(len(ends) - 1)
            pad = (-pos) % GROUP_ALIGN if gi + 1 < len(groups) else 0
            if pad:
                pos += pad
                ends.append(pos)
        gstart.append(pos)
        return pos, ends, gstart, rseg

    def _footprint(self, nbytes: int, nseg: int, cap: int):
        """(workspace bytes, region sizes..., total) of a batch: text, offsets, count, workspace, the
        (segment, offset, pattern_id) output, the pairs and the per-segment runs."""
        a = lambda x: (x + 255) // 256 * 256  # noqa: E731
        ws_bytes = self.automata[0].workspace_bytes(nbytes, nseg)
        sizes = [a(nbytes), a(8 * (nseg + 1)), 256, a(ws_bytes), a(12 * cap), a(8 * cap), a(8 * (nseg + 1))]
        return ws_bytes, sizes, sum(sizes)

    def _launch(self, groups, slot: _Slot, cap: int, fp):
        torch = self.torch
        nbytes, ends, gstart, rseg = self._layout(groups)
        nseg = len(ends)
        ws_bytes, sizes, total = fp
        got = self.arena.alloc(total)
        if got is None:
            return None
        off, ln = got
        offs = [off]
        for z in sizes[:-1]:
            offs.append(offs[-1] + z)
        t_off, s_off, c_off, w_off, m_off, p_off, f_off = offs
        b = _Batch()
        b.groups, b.slot, b.region, b.nbytes, b.cap = groups, slot, (off, ln), nbytes, cap
        b.reqs = [r for _, rs in groups for r in rs]
        b.nseg, b.gstart, b.rseg = nseg, np.array(gstart, np.uint64), rseg
        b.offsets = (t_off, s_off, c_off, w_off, m_off, p_off, f_off, ws_bytes)
        seg = slot.seg_host.numpy()
        seg[0] = 0
        seg[1:nseg + 1] = ends
        st = slot.stream
        with torch.cuda.stream(st):
            text = self.arena.view(t_off, nbytes)
            for gi, (si, rs) in enumerate(groups):
                a0 = int(gstart[gi])
                for r in rs:
                    n = r.payload.numel()
                    text[a0:a0 + n].copy_(r.payload, non_blocking=True)
                    a0 += n
                if a0 < gstart[gi + 1]:
                    text[a0:int(gstart[gi + 1])].zero_()
            self.arena.view(s_off, 8 * (nseg + 1)).view(torch.int64).copy_(slot.seg_host[:nseg + 1],
                                                                           non_blocking=True)
        self._scan_split(b, self.arena.base + m_off, self.arena.base + p_off, cap)
        b.copied = min(cap, slot.out_host.shape[0]) if cap <= self.EAGER_ROWS else 0
        with torch.cuda.stream(st):
            slot.count_host.copy_(self.arena.view(c_off, 8).view(torch.int64), non_blocking=True)
            slot.first_host[:nseg + 1].copy_(self.arena.view(f_off, 8 * (nseg + 1)).view(torch.int64),
                                             non_blocking=True)
            if b.copied:
                slot.out_host[:b.copied].copy_(self._pairs_view(b, b.copied), non_blocking=True)
        slot.ev.record(st)
        b.stage = 1
        return b

    def _scan_split(self, b, out_ptr: int, pairs_ptr: int, cap: int):
        t_off, s_off, c_off, w_off, m_off, p_off, f_off, ws_bytes = b.offsets
        base, st = self.arena.base, b.slot.stream.cuda_stream
        if len(b.groups) == 1:
            rc = self.lib.glop_scan_batch(self.automata[b.groups[0][0]].handle, base + t_off, b.nbytes,
                                          base + s_off, b.nseg, out_ptr, cap, base + c_off, base + w_off, ws_bytes,
                                          st)
        else:
            hs = (ctypes.c_void_p * len(b.groups))(*[self.automata[si].handle.value for si, _ in b.groups])
            rc = self.lib.glop_scan_batch_multi(hs, len(b.groups), b.gstart.ctypes.data, base + t_off, b.nbytes,
                                                base + s_off, b.nseg, out_ptr, cap, base + c_off, base + w_off,
                                                ws_bytes, st)
        if rc != OK:
            raise GlopError(rc, "glop_scan_batch")
        rc = self.lib.glop_batch_split(out_ptr, base + c_off, cap, b.nseg, pairs_ptr, base + f_off, st)
        if rc != OK:
            raise GlopError(rc, "glop_batch_split")

    def _pairs_view(self, b, n: int, start: int = 0):
        if b.slot.extra is not None:
            return b.slot.extra[1][start:n]
        p_off = b.offsets[5]
        return self.arena.view(p_off + 8 * start, 8 * (n - start)).view(self.torch.int32).view(-1, 2)

    def _advance(self, b):
        """Stage 1 done (count and runs on the host): rescan, fetch the remaining pairs, or finish."""
        torch = self.torch
        slot = b.slot
        total = int(slot.count_host.item())
        if total > b.cap:
            # the output bound was too small: scan the batch again into outputs of the true size
            self.stats["rescans"] += 1
            slot.extra = (torch.empty((total, 3), dtype=torch.int32, device=self.device),
                          torch.empty((total, 2), dtype=torch.int32, device=self.device))
            self._scan_split(b, slot.extra[0].data_ptr(), slot.extra[1].data_ptr(), total)
            b.cap, b.copied = total, 0
            f_off, nseg = b.offsets[6], b.nseg
            with torch.cuda.stream(slot.stream):  # the runs of the full output
                slot.first_host[:nseg + 1].copy_(self.arena.view(f_off, 8 * (nseg + 1)).view(torch.int64),
                                                 non_blocking=True)
        b.total = total
        if total > b.copied:
            host = slot.host_out(torch, total, keep=b.copied)
            with torch.cuda.stream(slot.stream):
                host[b.copied:total].copy_(self._pairs_view(b, total, b.copied), non_blocking=True)
            slot.ev.record(slot.stream)
            b.stage = 2
            return False
        return True

    def _finish(self, b, now: float):
        slot = b.slot
        pairs = slot.out_host[:b.total].numpy().view(np.uint32)
        first = slot.first_host[:b.nseg + 1].numpy()
        for r, k in zip(b.reqs, b.rseg):
            lo, hi = int(first[k]), int(first[k + 1])
            r.count = hi - lo
            if self.keep:
                r.matches = pairs[lo:hi].copy()
            r.done = now
        for si, rs in b.groups:
            nb = sum(r.payload.numel() for r in rs)
            self.density[si] = max(0.97 * self.density[si], sum(r.count for r in rs) / max(nb, 1))
        slot.extra = None
        self.arena.release(*b.region)
        self.stats["batches"] += 1
        self.stats["requests_per_batch_max"] = max(self.stats["requests_per_batch_max"], len(b.reqs))
        self.stats["sets_per_batch_max"] = max(self.stats.get("sets_per_batch_max", 0), len(b.groups))

    def _group(self, order, batched, r0):
        """The next batch: pending requests in arrival order, from the oldest one on, of every set whose
        automaton shares r0's kernel kind, within the batch limits; as groups (set, requests), by set."""
        kind = self.kind[r0.set_index]
        take, nbytes, by_set = [], 0, {}
        for r in order:
            if id(r) in batched or self.kind[r.set_index] != kind:
                continue
            sz = r.payload.numel()
            trial = dict(by_set)
            trial.setdefault(r.set_index, []).append(r)
            groups = sorted(trial.items())
            if take and (nbytes + sz > self.max_batch_bytes or len(take) >= self.max_batch_requests
                         or len(trial) > MAX_GROUPS or self._cap(groups) > self.out_rows):
                break
            take.append(r)
            by_set = trial
            nbytes += sz
        return sorted(by_set.items())

    # -- the loop --------------------------------------------------------------
    def serve(self, requests, realtime: bool = True):
        """Serve ``requests`` (sorted by arrival).  realtime: arrivals follow the trace's clock; else all
        requests are available at once (saturation).  Returns (wall seconds, stats of this call)."""
        import collections
        torch = self.torch
        self.stats = {"batches": 0, "rescans": 0, "requests_per_batch_max": 0, "admission_waits": 0, "fast": 0,
                      "big": 0}
        cnt = ctypes.c_uint64()
        big = self.big
        big_done0 = big.completed if big is not None else 0
        fifos = [collections.deque() for _ in self.automata]
        order = collections.deque()  # arrival order over all sets; requests already batched are skipped
        batched = set()
        inflight = []
        free_slots = list(self.slots)
        nxt = 0
        n = len(requests)
        t0 = time.perf_counter()
        if big is not None:
            big.t0 = t0
        done = 0
        n_big = 0
        while done + ((big.completed - big_done0) if big is not None else 0) < n:
            now = time.perf_counter() - t0
            while nxt < n and (not realtime or requests[nxt].arrival <= now):
                r = requests[nxt]
                if big is not None and r.payload.numel() >= self.big_bytes:
                    big.q.put(r)  # the large-request lane: no batch, no wait behind small ones
                    n_big += 1
                else:
                    fifos[r.set_index].append(r)
                    order.append(r)
                nxt += 1
            if big is not None and (big.error is not None or not big.thread.is_alive()):
                raise big.error or RuntimeError("the large-request lane stopped")
            progressed = False
            # completions
            for b in list(inflight):
                if not b.slot.ev.query():
                    continue
                progressed = True
                if b.stage == 1 and not self._advance(b):
                    continue
                self._finish(b, time.perf_counter() - t0)
                inflight.remove(b)
                free_slots.append(b.slot)
                done += len(b.reqs)
            # new batches while stream slots and device memory allow
            while free_slots:
                while order and id(order[0]) in batched:
                    batched.discard(id(order.popleft()))
                if not order:
                    break
                r0 = order[0]
                if (not inflight and len(order) == 1 and self.fast_bytes and
                        r0.payload.numel() <= self.fast_bytes):
                    rc = self.lib.glop_scan_host(self.automata[r0.set_index].handle, r0.payload.data_ptr(),
                                                 r0.payload.numel(), self.fast_out.data_ptr(), self.fast_cap,
                                                 ctypes.byref(cnt), self.fast_staging.data_ptr(),
                                                 self.fast_staging.numel(), self.fast_stream.cuda_stream)
                    if rc == OK:
                        r0.count = int(cnt.value)
                        if self.keep:
                            r0.matches = self.fast_out[:r0.count].numpy().view(np.uint32).copy()
                        r0.done = time.perf_counter() - t0
                        fifos[r0.set_index].popleft()
                        order.popleft()
                        done += 1
                        self.stats["fast"] += 1
                        progressed = True
                        continue
                    if rc != EOVERFLOW:
                        raise GlopError(rc, "glop_scan_host")
                    # more matches than the fast path holds: scan it as a batch
                groups = self._group(order, batched, r0)
                while True:
                    nb, ends, _, _ = self._layout(groups)
                    cap = self._cap(groups)
                    fp = self._footprint(nb, len(ends), cap)
                    if fp[2] <= self.arena.largest_free or sum(len(rs) for _, rs in groups) == 1:
                        break
                    # halve the batch: keep the older half of its requests
                    reqs = sorted((r for _, rs in groups for r in rs), key=lambda r: r.arrival)
                    keep = set(id(r) for r in reqs[:(len(reqs) + 1) // 2])
                    groups = [(si, [r for r in rs if id(r) in keep]) for si, rs in groups]
                    groups = [(si, rs) for si, rs in groups if rs]
                b = self._launch(groups, free_slots[-1], cap, fp)
                if b is None and not inflight:
                    # nothing else holds memory: try a minimal output (a larger one is made if needed)
                    b = self._launch(groups, free_slots[-1], 4096, self._footprint(nb, len(ends), 4096))
                if b is None:
                    self.stats["admission_waits"] += 1
                    if not inflight:
                        raise GlopError(2, "request of %d bytes does not fit the HBM budget" %
                                        groups[0][1][0].payload.numel())
                    break
                free_slots.pop()
                for si, rs in groups:  # (a batch takes the oldest pending requests of each of its sets)
                    for _ in rs:
                        fifos[si].popleft()
                batched.update(id(r) for _, rs in groups for r in rs)
                inflight.append(b)
                progressed = True
            if not progressed:
                if realtime and not inflight and not order and nxt < n:
                    time.sleep(max(0.0, min(requests[nxt].arrival - (time.perf_counter() - t0), 0.0005)))
                elif big is not None and (inflight or n_big):
                    time.sleep(0)  # let the lane's thread take the interpreter lock between its library calls
        torch.cuda.synchronize(self.device)
        self.stats["big"] = n_big
        if big is not None:
            self.stats["big_rescans"] = big.rescans
        return time.perf_counter() - t0, dict(self.stats)


class NativeServer:
    """The serving loop in native code (``glop_server_*``): the same policy as :class:`BatchServer` -- resident
    sets, HBM-budget admission, one launch over requests of several sets of a kernel kind, an idle fast path
    and a large-request lane -- run by the library, with results in pinned memory it pools.  This class only
    submits requests when they arrive, polls, and copies each result out."""

    def __init__(self, pattern_sets, hbm_budget: int = 8 << 30, max_inflight: int = 4,
                 max_batch_bytes: int = 256 << 20, max_batch_requests: int = 512, keep_matches: bool = False,
                 out_rows: int = 0, fast_bytes: int = 1 << 20, big_bytes: int = 8 << 20,
                 max_request_bytes: int = 0, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.automata = [Automaton(p) for p in pattern_sets]
        self.keep = keep_matches
        self.lib = lib()
        o = _ServerOpts(hbm_budget, max_inflight, max_batch_requests, max_batch_bytes, out_rows, fast_bytes,
                        big_bytes if max_request_bytes >= big_bytes > 0 else 0, max_request_bytes)
        hs = (ctypes.c_void_p * len(self.automata))(*[a.handle.value for a in self.automata])
        self._h = ctypes.c_void_p()
        rc = self.lib.glop_server_create(hs, len(self.automata), ctypes.byref(o), ctypes.byref(self._h))
        if rc != OK:
            raise GlopError(rc, "glop_server_create")
        self._res = (_ServerResult * 256)()

    def close(self):
        if self._h:
            self.lib.glop_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def stats(self) -> dict:
        st = _ServerStats()
        self.lib.glop_server_stats_get(self._h, ctypes.byref(st))
        return {k: int(getattr(st, k)) for k, _ in _ServerStats._fields_}

    def serve(self, requests, realtime: bool = True):
        """Serve ``requests`` (sorted by arrival; payloads pinned CPU uint8 tensors).  realtime: each request is
        submitted at its arrival time; else all at once.  Fills count, matches (when kept) and done (seconds
        from the start, the library's completion time).  Returns (wall seconds, stats)."""
        L, h = self.lib, self._h
        n = len(requests)
        by_id = {}
        nres = ctypes.c_uint32()
        t0 = time.perf_counter()
        t0_ns = time.monotonic_ns()
        nxt = done = 0
        before = self.stats()
        while done < n:
            now = time.perf_counter() - t0
            while nxt < n and (not realtime or requests[nxt].arrival <= now):
                r = requests[nxt]
                by_id[nxt] = r
                rc = L.glop_server_submit(h, nxt, r.set_index, r.payload.data_ptr() if r.payload.numel() else None,
                                          r.payload.numel())
                if rc != OK:
                    raise GlopError(rc, "glop_server_submit")
                nxt += 1
            if realtime and nxt < n:  # the library waits (and keeps the loop moving) until the next arrival
                wait = int(max(0.0, min(requests[nxt].arrival - (time.perf_counter() - t0), 2e-4)) * 1e6)
            else:
                wait = 200
            rc = L.glop_server_poll(h, self._res, len(self._res), ctypes.byref(nres), wait)
            if rc != OK:
                raise GlopError(rc, "glop_server_poll")
            for k in range(nres.value):
                res = self._res[k]
                r = by_id.pop(res.id)
                if res.status != OK:
                    raise GlopError(res.status, "request %d" % r.rid)
                r.count = int(res.count)
                if self.keep:
                    r.matches = (np.ctypeslib.as_array(ctypes.cast(res.matches, ctypes.POINTER(ctypes.c_uint32)),
                                                       shape=(2 * r.count,)).reshape(-1, 2).copy()
                                 if r.count else np.zeros((0, 2), np.uint32))
                r.done = (res.done_ns - t0_ns) / 1e9
                L.glop_server_release(h, res.id)
                done += 1
        wall = time.perf_counter() - t0
        after = self.stats()
        st = {k: after[k] - before[k] for k in ("batches", "fast", "big", "rescans", "admission_waits",
                                                 "pinned_allocs")}
        st["requests_per_batch_max"] = after["requests_per_batch_max"]
        st["sets_per_batch_max"] = after["sets_per_batch_max"]
        return wall, st


class PlainServer:
    """One request at a time in arrival order through the end-to-end glop_scan_host call."""

    def __init__(self, pattern_sets, max_request_bytes: int, keep_matches: bool = False, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.automata = [Automaton(p) for p in pattern_sets]
        self.keep = keep_matches
        self.cap = max(1 << 20, 2 * max_request_bytes)
        self.stream = torch.cuda.Stream(device=self.device)
        self._alloc(self.cap, max_request_bytes)
        self.lib = lib()
        self.stats = {"rescans": 0}

    def _alloc(self, cap: int, max_bytes: int):
        torch = self.torch
        need = ctypes.c_uint64()
        self.automata[0].handle  # noqa: B018
        lib().glop_scan_host_staging_size(self.automata[0].handle, max_bytes, cap, ctypes.byref(need))
        self.staging = torch.empty(int(need.value), dtype=torch.uint8, device=self.device)
        self.host_out = torch.empty((cap, 2), dtype=torch.int32, pin_memory=True)
        self.cap, self.max_bytes = cap, max_bytes

    def serve(self, requests, realtime: bool = True):
        t0 = time.perf_counter()
        cnt = ctypes.c_uint64()
        for r in requests:
            if realtime:
                wait = r.arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            n = r.payload.numel()
            while True:
                rc = self.lib.glop_scan_host(self.automata[r.set_index].handle, r.payload.data_ptr(), n,
                                             self.host_out.data_ptr(), self.cap, ctypes.byref(cnt),
                                             self.staging.data_ptr(), self.staging.numel(), self.stream.cuda_stream)
                if rc == EOVERFLOW:
                    self.stats["rescans"] += 1
                    self._alloc(int(cnt.value) + 1024, self.max_bytes)
                    continue
                if rc != OK:
                    raise GlopError(rc, "glop_scan_host")
                break
            r.count = int(cnt.value)
            if self.keep:
                r.matches = self.host_out[:r.count].numpy().view(np.uint32).copy()
            r.done = time.perf_counter() - t0
        return time.perf_counter() - t0, dict(self.stats)


def latency_summary(requests) -> dict:
    lat = np.array([r.done - r.arrival for r in requests]) * 1e3
    byt = sum(r.payload.numel() for r in requests)
    return {"requests": len(requests), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "max_ms": round(float(lat.max()), 3),
            "bytes": int(byt)}

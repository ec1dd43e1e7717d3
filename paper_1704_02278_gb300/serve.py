"""Continuous-batching scan server over device-resident automata.

The paper's use case (Sec. 1) pushes syslog traces and rules to a GPU server
that answers with the number and locations of suspect events; its library
streams the next batch of logs while a kernel runs (Sec. 6) and names
real-time operation as future work (Sec. 8).  This module is that serving
layer: several compiled pattern sets stay resident on the device, requests
(payload bytes + the set to scan with) arrive over time, and the loop

* admits a request when its payload, scratch and estimated output fit in a
  device-memory budget (an arena of one allocation, first-fit),
* batches the admitted requests of one pattern set into a single
  ``glop_scan_batch`` launch (one segment per request) while earlier batches
  are still on the GPU -- up to ``max_inflight`` batches overlap, each on its
  own stream, so copies of one batch run under the scan of another,
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

from . import Automaton, GlopError, lib, EOVERFLOW, OK


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
    """Per-stream resources reused by every batch the stream carries (no allocation per batch)."""

    def __init__(self, torch, device, max_requests: int):
        self.stream = torch.cuda.Stream(device=device)
        self.seg_host = torch.empty(max_requests + 1, dtype=torch.int64, pin_memory=True)
        self.count_host = torch.empty(1, dtype=torch.int64, pin_memory=True)
        self.out_host = torch.empty((1 << 16, 3), dtype=torch.int32, pin_memory=True)
        self.ev_count = torch.cuda.Event()
        self.ev_done = torch.cuda.Event()
        self.extra = None  # device output of a rescan

    def host_out(self, torch, n: int):
        if self.out_host.shape[0] < n:
            cap = max(n, 2 * self.out_host.shape[0])
            self.out_host = torch.empty((cap, 3), dtype=torch.int32, pin_memory=True)
        return self.out_host


class _Batch:
    pass


class BatchServer:
    """Continuous batching of scan requests over resident automata (see module doc)."""

    def __init__(self, pattern_sets, hbm_budget: int = 8 << 30, max_inflight: int = 4,
                 max_batch_bytes: int = 256 << 20, max_batch_requests: int = 512, keep_matches: bool = False,
                 device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.automata = [Automaton(p) for p in pattern_sets]
        self.arena = DeviceArena(hbm_budget, self.device)
        self.slots = [_Slot(torch, self.device, max_batch_requests) for _ in range(max_inflight)]
        self.max_inflight = max_inflight
        self.max_batch_bytes = max_batch_bytes
        self.max_batch_requests = max_batch_requests
        self.keep = keep_matches
        # matches per payload byte per set (running average); a batch whose output outgrows the estimate is
        # scanned again into a larger output
        self.density = [0.25] * len(self.automata)
        self.lib = lib()
        self.stats = {"batches": 0, "rescans": 0, "max_batch_requests": 0, "admission_waits": 0}

    # -- one batch -------------------------------------------------------------
    def _cap(self, si: int, nbytes: int) -> int:
        return int(self.density[si] * nbytes * 1.5) + 4096

    def _launch(self, reqs, set_index: int, slot: _Slot, cap: int):
        torch = self.torch
        nbytes = sum(r.payload.numel() for r in reqs)
        ws_bytes = self.automata[set_index].workspace_bytes(nbytes, len(reqs))
        t_len = (nbytes + 255) // 256 * 256
        s_len = (8 * (len(reqs) + 1) + 255) // 256 * 256
        got = self.arena.alloc(t_len + s_len + 256 + (ws_bytes + 255) // 256 * 256 + 12 * cap)
        if got is None:
            return None
        off, ln = got
        b = _Batch()
        b.reqs, b.set_index, b.slot, b.region, b.nbytes, b.cap = reqs, set_index, slot, (off, ln), nbytes, cap
        t_off = off
        s_off = t_off + t_len
        c_off = s_off + s_len
        w_off = c_off + 256
        m_off = w_off + (ws_bytes + 255) // 256 * 256
        seg = slot.seg_host.numpy()
        seg[0] = 0
        np.cumsum([r.payload.numel() for r in reqs], out=seg[1:len(reqs) + 1])
        b.seg = seg[:len(reqs) + 1].copy()
        st = slot.stream
        with torch.cuda.stream(st):
            text = self.arena.view(t_off, nbytes)
            for r, a0 in zip(reqs, b.seg[:-1]):
                text[int(a0):int(a0) + r.payload.numel()].copy_(r.payload, non_blocking=True)
            self.arena.view(s_off, 8 * (len(reqs) + 1)).view(torch.int64).copy_(slot.seg_host[:len(reqs) + 1],
                                                                                  non_blocking=True)
        rc = self.lib.glop_scan_batch(self.automata[set_index].handle, self.arena.base + t_off, nbytes,
                                      self.arena.base + s_off, len(reqs), self.arena.base + m_off, cap,
                                      self.arena.base + c_off, self.arena.base + w_off, ws_bytes, st.cuda_stream)
        if rc != OK:
            self.arena.release(off, ln)
            raise GlopError(rc, "glop_scan_batch")
        with torch.cuda.stream(st):
            slot.count_host.copy_(self.arena.view(c_off, 8).view(torch.int64), non_blocking=True)
        slot.ev_count.record(st)
        b.offsets = (t_off, s_off, c_off, w_off, m_off, ws_bytes)
        b.stage = 1
        return b

    def _fetch(self, b, total: int):
        torch = self.torch
        slot = b.slot
        t_off, s_off, c_off, w_off, m_off, ws_bytes = b.offsets
        if total > b.cap:
            # the output bound was too small: scan this batch again into a larger output
            self.stats["rescans"] += 1
            slot.extra = torch.empty((total, 3), dtype=torch.int32, device=self.device)
            rc = self.lib.glop_scan_batch(self.automata[b.set_index].handle, self.arena.base + t_off, b.nbytes,
                                          self.arena.base + s_off, len(b.reqs), slot.extra.data_ptr(), total,
                                          self.arena.base + c_off, self.arena.base + w_off, ws_bytes,
                                          slot.stream.cuda_stream)
            if rc != OK:
                raise GlopError(rc, "glop_scan_batch")
            dev_out = slot.extra
        else:
            dev_out = self.arena.view(m_off, 12 * total).view(torch.int32).view(total, 3) if total else None
        host = slot.host_out(torch, max(total, 1))
        if total:
            with torch.cuda.stream(slot.stream):
                host[:total].copy_(dev_out, non_blocking=True)
        slot.ev_done.record(slot.stream)
        b.total = total
        b.stage = 2

    def _finish(self, b, now: float):
        slot = b.slot
        m = slot.out_host[:b.total].numpy().view(np.uint32) if b.total else np.zeros((0, 3), np.uint32)
        bounds = np.searchsorted(m[:, 0], np.arange(len(b.reqs) + 1))
        for k, r in enumerate(b.reqs):
            lo, hi = bounds[k], bounds[k + 1]
            r.count = int(hi - lo)
            if self.keep:
                r.matches = m[lo:hi, 1:].copy()
            r.done = now
        self.density[b.set_index] = 0.8 * self.density[b.set_index] + 0.2 * (b.total / max(b.nbytes, 1))
        slot.extra = None
        self.arena.release(*b.region)
        self.stats["batches"] += 1
        self.stats["max_batch_requests"] = max(self.stats["max_batch_requests"], len(b.reqs))

    # -- the loop --------------------------------------------------------------
    def serve(self, requests, realtime: bool = True):
        """Serve ``requests`` (sorted by arrival).  realtime: arrivals follow the trace's clock; else all
        requests are available at once (saturation).  Returns (wall seconds, stats)."""
        torch = self.torch
        pending = []
        inflight = []
        free_slots = list(self.slots)
        nxt = 0
        n = len(requests)
        t0 = time.perf_counter()
        done = 0
        while done < n:
            now = time.perf_counter() - t0
            while nxt < n and (not realtime or requests[nxt].arrival <= now):
                pending.append(requests[nxt])
                nxt += 1
            progressed = False
            # completions
            for b in list(inflight):
                if b.stage == 1 and b.slot.ev_count.query():
                    self._fetch(b, int(b.slot.count_host.item()))
                    progressed = True
                if b.stage == 2 and b.slot.ev_done.query():
                    self._finish(b, time.perf_counter() - t0)
                    inflight.remove(b)
                    free_slots.append(b.slot)
                    done += len(b.reqs)
                    progressed = True
            # new batches while stream slots and device memory allow
            while pending and free_slots:
                si = pending[0].set_index
                group, nbytes = [], 0
                for r in pending:
                    if r.set_index != si:
                        continue
                    sz = r.payload.numel()
                    if group and (nbytes + sz > self.max_batch_bytes or len(group) >= self.max_batch_requests):
                        break
                    group.append(r)
                    nbytes += sz
                b = self._launch(group, si, free_slots[-1], self._cap(si, nbytes))
                if b is None and len(group) > 1:
                    group = group[:1]
                    b = self._launch(group, si, free_slots[-1], self._cap(si, group[0].payload.numel()))
                if b is None and not inflight:
                    # nothing else holds memory: try a minimal output (a larger one is made if needed)
                    b = self._launch(group, si, free_slots[-1], 4096)
                if b is None:
                    self.stats["admission_waits"] += 1
                    if not inflight:
                        raise GlopError(2, "request of %d bytes does not fit the HBM budget" %
                                        group[0].payload.numel())
                    break
                free_slots.pop()
                if len(group) == len(pending):
                    pending = []
                else:
                    ids = {id(r) for r in group}
                    pending = [r for r in pending if id(r) not in ids]
                inflight.append(b)
                progressed = True
            if not progressed:
                if realtime and not inflight and not pending and nxt < n:
                    time.sleep(max(0.0, min(requests[nxt].arrival - (time.perf_counter() - t0), 0.0005)))
        torch.cuda.synchronize(self.device)
        return time.perf_counter() - t0, dict(self.stats)


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

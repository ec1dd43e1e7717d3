#!/usr/bin/env python
"""Benchmark: Gbit/s scanned (Eq. 1: 8 * N / time) by the GB300 multi-pattern scan.

Default workload: 256 MiB of seeded synthetic syslog text (2 % of lines carry a
planted pattern) against 1,000 patterns of 4..64 bytes, 10 % of them
prefixes of others.  A step is one full scan of the buffer -- every offset
walked, every match written sorted to device memory, count included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

One JSON line on stdout (rank 0).  Under torchrun each rank scans its own copy
of the workload (independent shards, no collective): weak scaling.
``--impl reference`` times the CPU oracle (multi-threaded Aho-Corasick) on
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SMS = 152           # streaming multiprocessors of a GB300
CHUNK = 31 * 1024    # text bytes one block stages at a time (31 sub-tiles)
SUBTILE = 1024      # bytes per warp work unit (16-byte status record each)


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("scan_kernel.cuh", "scan.cu")  # the scan kernel and its launcher


def kernel_sha() -> str:
    """sha256 prefix of the scan kernel's sources, as the committed ncu summaries record it."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1704_02278_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_value(workload: str, kind: str, key: str):
    """An integer ``key: N`` from the committed ncu summary profiles/scan_kernel_<workload>_<kind>.md, when
    it was taken on the current kernel sources (their sha256 prefix matches); else None."""
    import re
    path = os.path.join(ROOT, "profiles", "scan_kernel_%s_%s.md" % (workload, kind))
    try:
        txt = open(path).read()
        sha = kernel_sha()
    except OSError:
        return None
    m_sha = re.search(r"kernel sources sha256 prefix: ([0-9a-f]{16})", txt)
    m_v = re.search(re.escape(key) + r": (\d+)", txt)
    if not m_sha or not m_v or m_sha.group(1) != sha:
        return None
    return int(m_v.group(1))


def profiled_traffic(workload: str):
    """DRAM bytes (read + write) per scan-kernel launch from the committed ncu summary of this workload,
    when it was taken on the current kernel sources; else None."""
    return profiled_value(workload, "traffic", "traffic_bytes_per_launch")


def read_stream_peak(dev, nbytes: int = 4 << 30, reps: int = 10):
    """Read-only HBM bandwidth on this GPU now: a sum over an int64 buffer larger than L2 (GB/s)."""
    import torch
    x = torch.ones(nbytes // 8, dtype=torch.int64, device=dev)
    for _ in range(3):
        x.sum()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        x.sum()
    e1.record()
    torch.cuda.synchronize()
    gbs = nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
    del x
    torch.cuda.empty_cache()
    return round(gbs, 1)


def link_roofline(host, staging, hm_pinned, N: int, M: int, step_s: float, reps: int = 10):
    """The host link's floor for one end-to-end step: plain copies of the step's bytes (the text up from the
    same pinned buffer, the matches down into the same pinned buffer), each alone and both at once on two
    streams; frac = that floor / the measured end-to-end step."""
    import torch
    dev = staging.device
    up_s, down_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    d_text = staging[:N]
    d_out = staging[N:N + 8 * M] if staging.numel() >= N + 8 * M else torch.empty(8 * M, dtype=torch.uint8, device=dev)
    h_out = hm_pinned.view(torch.uint8).reshape(-1)[:8 * M]

    def up():
        with torch.cuda.stream(up_s):
            d_text.copy_(host[:N], non_blocking=True)

    def down():
        with torch.cuda.stream(down_s):
            h_out.copy_(d_out, non_blocking=True)

    def both():
        up()
        down()

    def timed(fn):
        best = float("inf")
        for _ in range(3):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            best = min(best, (time.perf_counter() - t0) / reps)
        return best

    tu, td, tb = timed(up), timed(down), timed(both)
    return {"h2d_GBps": round(N / tu / 1e9, 1), "d2h_GBps": round(8 * M / td / 1e9, 1),
            "h2d_ms": round(tu * 1e3, 3), "d2h_ms": round(td * 1e3, 3), "both_ms": round(tb * 1e3, 3),
            "e2e_ms": round(step_s * 1e3, 3), "frac": round(tb / step_s, 4),
            "note": "plain cudaMemcpyAsync of the step's bytes from/to the same pinned buffers (best of 3 x %d); "
                    "frac = both copies at once / end-to-end step" % reps}


def walk_stats(w, sample_bytes: int = 8 << 20):
    """Walk counters of the scan's decision rules on the first sample_bytes of the workload (whole
    segments for batches), from the library's host walk emulation: start-filter pass rate, gram-table
    hits, and the table lookups a walk makes past its gram (E[depth])."""
    import ctypes
    from paper_1704_02278_gb300 import _build
    L = ctypes.CDLL(_build.build_hostcheck())
    L.glop_hostcheck_set_options(ctypes.c_uint32(0), ctypes.c_uint32(0))
    if w.seg is None:
        n = min(sample_bytes, w.text.size)
        seg = np.array([0, n], np.uint64)
    else:
        k = int(np.searchsorted(w.seg, sample_bytes, side="right"))
        seg = np.ascontiguousarray(w.seg[:max(k, 2)], dtype=np.uint64)
        n = int(seg[-1])
    text = np.ascontiguousarray(w.text[:n])
    pb = np.ascontiguousarray(w.patterns.buf, np.uint8)
    po = np.ascontiguousarray(w.patterns.offs, np.uint64)
    out = ctypes.POINTER(ctypes.c_uint32)()
    cnt = ctypes.c_uint64()
    st = np.zeros(16, np.uint64)
    vp = ctypes.c_void_p
    rc = L.glop_hostcheck_scan(vp(pb.ctypes.data), vp(po.ctypes.data), ctypes.c_uint32(len(po) - 1),
                               ctypes.c_uint32(0), vp(text.ctypes.data), vp(seg.ctypes.data),
                               ctypes.c_uint32(len(seg) - 1), ctypes.byref(out), ctypes.byref(cnt),
                               vp(st.ctypes.data))
    if rc:
        return None
    if cnt.value:
        L.glop_hostcheck_free(out)
    n_states, n_dense, n_classes, gram, passed, found, dense, chain_in, chain_b, matched = [int(v) for v in st[:10]]
    walks = max(found, 1)
    return {"sample_bytes": n, "gram_len": gram, "filter_pass_per_offset": round(passed / n, 4),
            "gram_hits_per_offset": round(found / n, 4), "matched_offsets_per_offset": round(matched / n, 4),
            "dense_steps_per_walk": round(dense / walks, 3), "chain_pieces_per_walk": round(chain_in / walks, 3),
            "chain_bytes_per_walk": round(chain_b / walks, 3),
            "E_depth": round(gram + (dense + chain_b) / walks, 3),
            "E_depth_note": "mean bytes a walk examines from its start offset: the gram, then one per dense step "
                            "and every chain byte compared (the mismatching one included)",
            "lookups_per_offset": round((n + found + dense + chain_in) / n, 4),
            "source": "host walk emulation (same decision rules), sample of the workload"}


def verify_output(w, matches, M: int, sample_bytes: int = 64 << 20):
    """Compare the scan output left in ``matches`` by the timed steps with the oracle.  Single buffer: the
    whole (offset, pattern_id) list against the multi-threaded Aho-Corasick oracle.  Batches: every segment
    that starts in the first ``sample_bytes`` of the buffer, against the oracle's per-segment scan of those
    segments (the oracle is too slow for all of config 3 or 4 within the bench's minutes)."""
    import oracle
    import torch
    t0 = time.perf_counter()
    if w.seg is None:
        got = matches[:M].cpu().numpy().view(np.uint32)
        exp = oracle.ac_mt(w.text, w.patterns.csr())
        ok = bool(len(exp) == M and np.array_equal(got, exp))
        what = "all %d matches vs oracle.ac_mt on the whole text" % M
    else:
        k = int(np.searchsorted(w.seg, sample_bytes, side="right"))
        k = max(1, min(k, len(w.seg) - 1))
        seg = np.ascontiguousarray(w.seg[:k + 1], dtype=np.uint64)
        exp = oracle.batch(w.text[:int(seg[-1])], seg, w.patterns.csr())
        col = matches[:M, 0].contiguous()
        n = int(torch.searchsorted(col, torch.tensor([k], dtype=col.dtype, device=col.device)).item())
        del col
        got = matches[:n].cpu().numpy().view(np.uint32)
        ok = bool(n == len(exp) and np.array_equal(got, exp))
        what = "segments 0..%d (%d bytes, %d matches) vs oracle.batch" % (k - 1, int(seg[-1]), len(exp))
    return {"ok": ok, "checked": what, "seconds": round(time.perf_counter() - t0, 2)}


def make_workload(name: str):
    import workloads as W
    if name == "syslog-256MiB-1000pat":
        return W.config2()
    if name == "syslog-1MiB-100pat":
        return W.config1()
    if name == "dpi-2GiB-20000sig":
        return W.config3()
    if name == "files-10000-5000pat":
        return W.config4()
    if name.startswith("syslog-") and name.endswith("MiB-1000pat"):
        return W.config2(int(name.split("-")[1][:-3]) * W.MiB)
    if name.startswith("dpi-") and name.endswith("MiB-20000sig"):
        return W.config3(int(name.split("-")[1][:-3]) * W.MiB)
    raise SystemExit("unknown workload " + name)


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the GPU works."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        time.sleep(0.05)
        return self.summary()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args, ws, rank):
    """The CPU oracle on this host's cores, on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    w = make_workload(args.workload)
    cores = os.cpu_count() or 1
    pats = w.patterns.csr()
    # each step is a bounded sample, sized from a 4 MiB calibration run so that warm-up and timed steps
    # together take about two minutes (at most --ref-sample-mib MiB per step)
    cal = w.text[: min(w.nbytes, 4 << 20)]
    t0 = time.perf_counter()
    oracle.ac_mt(cal, pats, threads=cores)
    rate = cal.size / max(time.perf_counter() - t0, 1e-6)
    per_step = 120.0 / max(args.steps + args.warmup, 1)
    nbytes = int(min(args.ref_sample_mib << 20, max(256 << 10, rate * per_step)))
    sample = w.text[: min(w.nbytes, nbytes)]
    for _ in range(args.warmup):
        oracle.ac_mt(sample, pats, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.ac_mt(sample, pats, threads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    gbps = 8.0 * sample.size * len(times) / tot / 1e9
    line = {
        "impl": "reference", "metric": "Gbit/s scanned (8*N/t, Eq. 1)", "value": round(gbps, 4),
        "unit": "Gbit/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / len(times), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "sample_bytes": int(sample.size)},
        "cpu_baseline": {"value": round(gbps, 4), "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                         "sample": "first %.2f MiB of the workload per step (%s), multi-threaded Aho-Corasick "
                                   "oracle" % (sample.size / 2**20,
                                               "sized so all %d steps take about two minutes" % args.steps
                                               if sample.size < min(w.nbytes, args.ref_sample_mib << 20) else
                                               "the %d MiB cap per step" % (min(w.nbytes, args.ref_sample_mib << 20)
                                                                            >> 20))},
        "e2e": {"value": round(gbps, 4), "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(w, budget_s: float = 20.0):
    """The oracle as it stands on all host cores over a bounded sample of the workload: the best of at
    least three runs (the host is shared, so single runs vary)."""
    import oracle
    cores = os.cpu_count() or 1
    pats = w.patterns.csr()
    n = min(w.nbytes, 64 << 20)
    sample = w.text[:n]
    times = []
    spent = 0.0
    while len(times) < 3 or (spent < budget_s / 4 and len(times) < 8):
        t0 = time.perf_counter()
        oracle.ac_mt(sample, pats, threads=cores)
        times.append(time.perf_counter() - t0)
        spent += times[-1]
        if spent > budget_s:
            break
    out = {"value": round(8.0 * n / min(times) / 1e9, 4), "unit": "Gbit/s", "cores": cores, "kind": "oracle",
           "sample": "first %d MiB of the workload, best of %d runs (median %.4f Gbit/s), multi-threaded "
                     "Aho-Corasick oracle" % (n >> 20, len(times), 8.0 * n / statistics.median(times) / 1e9)}
    # the same oracle on one thread, over a smaller sample
    n1 = min(w.nbytes, 8 << 20)
    t0 = time.perf_counter()
    oracle.ac(w.text[:n1], pats)
    out["single_thread"] = {"value": round(8.0 * n1 / (time.perf_counter() - t0) / 1e9, 4), "unit": "Gbit/s",
                            "sample": "first %d MiB, one run, Aho-Corasick oracle on one thread" % (n1 >> 20)}
    # the naive every-pattern-at-every-offset oracle, on the small configuration only
    if w.nbytes <= (1 << 20):
        t0 = time.perf_counter()
        oracle.naive(w.text, pats)
        out["naive"] = {"value": round(8.0 * w.nbytes / (time.perf_counter() - t0) / 1e9, 4), "unit": "Gbit/s",
                        "sample": "the whole %d-byte text, one run, one thread" % w.nbytes}
    return out


def run_prefix_fp(args, ws, rank):
    """False positives of the paper's 8-byte prefix matching (Sec. 5): every pattern cut to its first
    8 bytes reports a superset of the exact matches; the extra reports are the false positives."""
    if rank != 0:
        return
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_02278_gb300 as glop
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    res = {}
    for name, w in (("syslog-256MiB-1000pat", W.config2()), ("dpi-2GiB-20000sig", W.config3())):
        text = torch.from_numpy(w.text).to(dev)
        seg = None if w.seg is None else torch.from_numpy(w.seg.view(np.int64).copy()).to(dev)
        row = {}
        for k in (0, 8):
            a = glop.Automaton(w.patterns, prefix_len=k)
            if seg is None:
                m, n = a.scan(text)
                run = lambda: a.scan_into(text, m, cnt)  # noqa: E731
            else:
                m, n = a.scan_batch(text, seg)
                run = lambda: a.scan_batch_into(text, seg, m, cnt)  # noqa: E731
            cnt = torch.zeros(1, dtype=torch.int64, device=dev)
            for _ in range(3):
                run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                run()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 10
            row["exact" if k == 0 else "prefix8"] = {"matches": int(n), "ms": round(ms, 4),
                                                     "gbps": round(8.0 * w.nbytes / ms / 1e6, 1)}
            del m
            a.close()
            torch.cuda.empty_cache()
        ex, pr = row["exact"]["matches"], row["prefix8"]["matches"]
        row["false_positives"] = pr - ex
        row["fp_rate"] = (pr - ex) / pr if pr else 0.0
        res[name] = row
        del text
        torch.cuda.empty_cache()
    line = {"metric": "false-positive rate of 8-byte prefix matching (false reports / prefix-mode reports)",
            "value": res["syslog-256MiB-1000pat"]["fp_rate"], "unit": "fraction", "n_gpus": 1, "steps": 10,
            "warmup": 3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": "prefix8-fp (configs 2 and 3)"}, "prefix_fp": res}
    print(json.dumps(line), flush=True)


def run_stream(args, ws, rank):
    """Streaming ingestion of config 2 (256 MiB syslog, 1,000 patterns) from pinned host memory in 16 MiB
    chunks: the StreamScanner (three slots: upload and scan of one chunk under the copy-back of the previous
    one; halo carried on the device), against its two-slot form and against the same chunks scanned one after
    another through glop_scan_host."""
    if rank != 0:
        return
    import ctypes
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_02278_gb300 as glop
    from paper_1704_02278_gb300.stream import StreamScanner
    import workloads as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = W.config2()
    N = w.nbytes
    chunk = 16 << 20
    host = torch.from_numpy(w.text).pin_memory()
    chunks = [host[i:i + chunk] for i in range(0, N, chunk)]
    a = glop.Automaton(w.patterns)

    def timed_stream(depth):
        sc = StreamScanner(a, chunk_bytes=chunk, out_rows=8 << 20, depth=depth)

        def streamed():
            n = 0
            for c in chunks:
                n += len(sc.feed(c))
            return n + sum(len(r) for r in sc.flush())

        m = streamed()
        times = []
        for _ in range(max(args.steps, 3)):
            sc.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            assert streamed() == m
            times.append(time.perf_counter() - t0)
        sc.close()
        return m, times

    M, times = timed_stream(2)
    M1, times1 = timed_stream(1)
    assert M1 == M
    # the same chunks, one glop_scan_host call after another (each copies in, scans and copies back)
    halo = a.info["max_pattern_len"] - 1
    need = ctypes.c_uint64()
    cap = 8 << 20
    glop.lib().glop_scan_host_staging_size(a.handle, chunk + halo, cap, ctypes.byref(need))
    staging = torch.empty(int(need.value), dtype=torch.uint8, device=dev)
    hout = torch.empty((cap, 2), dtype=torch.int32, pin_memory=True)
    cnt = ctypes.c_uint64()
    st = torch.cuda.Stream()
    ser = []
    for _ in range(max(args.steps, 3)):
        t0 = time.perf_counter()
        for i in range(0, N, chunk):
            lo = max(0, i - halo)
            rc = glop.lib().glop_scan_host(a.handle, host.data_ptr() + lo, min(N, i + chunk) - lo, hout.data_ptr(),
                                           cap, ctypes.byref(cnt), staging.data_ptr(), staging.numel(),
                                           st.cuda_stream)
            assert rc == 0, rc
        ser.append(time.perf_counter() - t0)
    tm, ts, t1 = statistics.median(times), statistics.median(ser), statistics.median(times1)
    line = {"metric": "Gbit/s ingested from a host stream (8*N/t, Eq. 1)", "value": round(8.0 * N / tm / 1e9, 3),
            "unit": "Gbit/s", "n_gpus": 1, "steps": len(times), "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "stream-256MiB-1000pat", "chunk_bytes": chunk, "matches": int(M)},
            "stream": {"depth": 2, "depth2_s": round(tm, 4), "depth1_s": round(t1, 4),
                       "depth1_gbps": round(8.0 * N / t1 / 1e9, 3), "serial_glop_scan_host_s": round(ts, 4),
                       "serial_gbps": round(8.0 * N / ts / 1e9, 3),
                       "note": "timed from the first chunk fed to the last match in host memory (the owned rows of each "
                "chunk, pinned, relative to the chunk's base)"}}
    print(json.dumps(line), flush=True)


def serve_record(seconds: float, hbm_gib: int, saturated_runs: int = 3):
    """Serving trace (Poisson arrivals at 200 req/s, log-normal sizes, 8 resident sets): plain per-request
    scans vs continuous batching, in real time (latency) and saturated (throughput).  Returns the record."""
    import torch
    import workloads as W
    from paper_1704_02278_gb300 import serve
    sets = W.config5_sets()
    times, sizes, set_idx = W.config5_requests(200.0, float(seconds))
    pool_bytes = 256 << 20
    pools = [torch.from_numpy(W.config5_payload(k, pool_bytes)).pin_memory() for k in (0, 1)]

    def make():
        reqs = []
        for i in range(len(times)):
            size = int(min(sizes[i], pool_bytes))
            off = (i * 2654435761) % (pool_bytes - size + 1)
            reqs.append(serve.Request(i, int(set_idx[i]), pools[i % 2][off:off + size], float(times[i])))
        return reqs

    out = {"requests": len(times), "bytes": int(sizes.sum()), "seconds": seconds}
    plain = serve.PlainServer(sets, max_request_bytes=int(sizes.max()))
    # pinned result buffers sized for a full 256 MiB batch at up to 0.25 matches per byte
    # requests of 8 MiB and more go to the large-request lane, sized like the plain server's buffers
    # (a lone request of up to 8 MiB on an idle server takes one end-to-end call, as the plain loop does;
    # larger ones take the lane)
    batched = serve.BatchServer(sets, hbm_budget=hbm_gib << 30, out_rows=(256 << 20) // 4,
                                max_request_bytes=int(sizes.max()), fast_bytes=8 << 20)
    # the same policy with the loop in native code (glop_server_*)
    native = serve.NativeServer(sets, hbm_budget=hbm_gib << 30, out_rows=(256 << 20) // 4,
                                max_request_bytes=int(sizes.max()), fast_bytes=8 << 20)
    # warm all three (first launches, host allocator)
    plain.serve(make()[:20], realtime=False)
    batched.serve(make()[:20], realtime=False)
    native.serve(make()[:20], realtime=False)
    for name, srv in (("plain", plain), ("batched", batched), ("native", native)):
        reqs = make()
        wall, st = srv.serve(reqs, realtime=True)
        lat = serve.latency_summary(reqs)
        # saturation: every request available at once; several runs (the host loop is sensitive to the
        # shared host's load), median reported, best kept beside it
        walls = []
        for _ in range(saturated_runs):
            reqs2 = make()
            wall2, st2 = srv.serve(reqs2, realtime=False)
            walls.append(wall2)
        wmed = statistics.median(walls)
        out[name] = dict(lat, realtime_wall_s=round(wall, 3), realtime_stats=st, saturated_s=round(wmed, 3),
                         saturated_gbps=round(8.0 * out["bytes"] / wmed / 1e9, 3),
                         saturated_gbps_best=round(8.0 * out["bytes"] / min(walls) / 1e9, 3),
                         saturated_runs=len(walls), stats=st2, matches=int(sum(r.count for r in reqs2)))
    batched.close()
    native.close()
    del plain, batched, native, pools
    torch.cuda.empty_cache()
    return out


def run_serve(args, ws, rank):
    """The serving trace alone (config 5), for --serve-seconds of arrivals."""
    if rank != 0:
        return
    import torch
    import __graft_entry__
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    out = serve_record(args.serve_seconds, args.serve_hbm_gib)
    line = {"metric": "served p50/p99 latency (ms) and saturated Gbit/s: continuous batching vs plain",
            "value": out["native"]["saturated_gbps"], "unit": "Gbit/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "serve-200rps-%ds-8sets" % args.serve_seconds,
                       "value_arm": "native serving loop (glop_server_*), saturated"}, "serve": out}
    print(json.dumps(line), flush=True)


def dpi_record(dev, steps: int, warmup: int, local: int):
    """The 20,000-signature point (config 3): 2 GiB of packets scanned as one batch, each step one replay of
    the captured scan (a single CUDA-graph launch), device-resident input, CUDA events on the launching
    stream; the timed output is checked against the oracle on a sample of whole packets."""
    import torch
    import paper_1704_02278_gb300 as glop
    w = make_workload("dpi-2GiB-20000sig")
    N = w.nbytes
    text = torch.from_numpy(w.text).to(dev)
    seg = torch.from_numpy(w.seg.view(np.int64).copy()).to(dev)
    a = glop.Automaton(w.patterns)
    stream = torch.cuda.Stream(device=dev)
    m0, M = a.scan_batch(text, seg, stream=stream)
    del m0
    torch.cuda.empty_cache()
    matches = torch.empty((max(M, 1), 3), dtype=torch.int32, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    plan = glop.Plan(a, text, matches, count, seg_offsets=seg, stream=stream)
    clocks = ClockSampler(local).start()
    for _ in range(warmup):
        plan.launch(stream)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        e0.record(stream)
        plan.launch(stream)
        e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    per = [e0.elapsed_time(e1) for e0, e1 in ev]
    st = a.status(dev, stream=stream, batch=True)
    assert st == glop.OK, "scan status %s" % glop.STATUS.get(st)
    assert int(count.item()) == M
    verified = verify_output(w, matches, M)
    ms = statistics.mean(per)
    hbm, which = peaks()
    halo = a.info["max_pattern_len"]
    n_chunks = (N + CHUNK - 1) // CHUNK
    n_tiles = (N + SUBTILE - 1) // SUBTILE
    algo_bytes = N + n_chunks * min(max(halo - 1, 16), 1024) + 12 * M + 16 * n_tiles
    achieved = algo_bytes / (ms / 1e3) / 1e9
    rec = {"workload": "dpi-2GiB-20000sig", "text_bytes": N, "segments": int(len(w.seg) - 1),
           "patterns": w.patterns.n, "matches": M, "steps": steps, "warmup": warmup,
           "ms_per_step": round(ms, 4), "median_ms": round(statistics.median(per), 4),
           "value": round(8.0 * N / (ms / 1e3) / 1e9, 3), "unit": "Gbit/s",
           "launch": "cuda graph (memset + init + scan kernel) per step", "gpu_launches": 2 * steps,
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(achieved / hbm, 4), "traffic": profiled_traffic("dpi-2GiB-20000sig"),
                        "note": "algorithmic bytes = text + halo re-reads + 12 B/match + tile status; peak %s"
                                % which},
           "hbm_input_frac": round(N / (ms / 1e3) / 1e9 / hbm, 4),
           "verified": verified["ok"], "verification": verified, "clocks": clk}
    ins = profiled_value("dpi-2GiB-20000sig", "traffic", "inst_per_launch")
    if ins is not None:
        f_sm = (clk or {}).get("sm_mhz") or 2070.0
        peak_issue = 4 * SMS * f_sm * 1e6
        rec["issue_roofline"] = {"bound": "issue", "achieved": round(ins / (ms / 1e3) / 1e12, 4),
                                 "peak": round(peak_issue / 1e12, 4), "unit": "T warp-instructions/s",
                                 "frac": round(ins / (ms / 1e3) / peak_issue, 4), "inst_per_launch": ins}
    del plan, matches, text, seg, count
    a.close()
    torch.cuda.empty_cache()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="syslog-256MiB-1000pat")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--ref-sample-mib", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the read-stream peak, walk statistics and count-only timing")
    ap.add_argument("--per-segment-steps", type=int, default=1)
    ap.add_argument("--serve-seconds", type=int, default=60)
    ap.add_argument("--extra-serve-seconds", type=int, default=20,
                    help="arrival seconds of the serving trace replayed for the default line's serve record")
    ap.add_argument("--dpi-steps", type=int, default=50)
    ap.add_argument("--serve-hbm-gib", type=int, default=16)
    ap.add_argument("--smem-budget", type=int, default=0,
                    help="shared-memory bytes for dense rows (0: automatic; 1: none, rows read through L1/L2)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload.startswith("serve"):
        run_serve(args, ws, rank)
        return
    if args.workload == "prefix8-fp":
        run_prefix_fp(args, ws, rank)
        return
    if args.workload == "stream-256MiB-1000pat":
        run_stream(args, ws, rank)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_02278_gb300 as glop

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    w = make_workload(args.workload)
    N = w.nbytes
    import hashlib
    text_sha = hashlib.sha256(memoryview(np.ascontiguousarray(w.text))).hexdigest()  # logged with the line
    host = torch.empty(N, dtype=torch.uint8, pin_memory=True)
    host.numpy()[:] = w.text
    text = host.to(dev)
    seg = None
    if w.seg is not None:
        seg = torch.from_numpy(w.seg.view(np.int64).copy()).to(dev)
    # (--smem-budget 1 keeps every dense row in L1/L2: the on-chip-table ablation)
    a = glop.Automaton(w.patterns, smem_budget=args.smem_budget)
    stream = torch.cuda.Stream(device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    # size the output once (the count does not change between steps)
    if seg is None:
        m0, M = a.scan(text, stream=stream)
    else:
        m0, M = a.scan_batch(text, seg, stream=stream)
    rec = 2 if seg is None else 3
    del m0
    torch.cuda.empty_cache()
    matches = torch.empty((max(M, 1), rec), dtype=torch.int32, device=dev)
    ws_buf = a.workspace(N, dev, None if seg is None else w.seg.size - 1)
    plan = None
    if seg is not None:
        # a batch step is one replay of the captured scan: a single graph launch over every segment
        plan = glop.Plan(a, text, matches, count, seg_offsets=seg, stream=stream)

    def step():
        if plan is not None:
            plan.launch(stream)
        else:
            a.scan_into(text, matches, count, workspace=ws_buf, stream=stream)

    clocks = ClockSampler(local).start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for i in range(args.steps):
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    t_all1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    total_ms = t_all0.elapsed_time(t_all1)
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    st = a.status(dev, stream=stream, batch=seg is not None)
    assert st == glop.OK, "scan status %s" % glop.STATUS.get(st)
    assert int(count.item()) == M
    # the match list the timed steps wrote, compared element by element with the CPU oracle (outside the
    # timed region): the whole list for a single buffer; for batches a sample of whole segments
    verified = verify_output(w, matches, M)

    t_max = total_ms
    if pg:
        tt = torch.tensor([total_ms], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_max = float(tt.item())
    gbps = 8.0 * N * args.steps * ws / (t_max / 1e3) / 1e9

    # roofline of the scan (init + scan kernel per launch; the init kernel clears ~N/4096 words)
    hbm, which = peaks()
    halo = a.info["max_pattern_len"]
    n_chunks = (N + CHUNK - 1) // CHUNK
    n_tiles = (N + SUBTILE - 1) // SUBTILE
    algo_bytes = N + n_chunks * min(max(halo - 1, 16), 1024) + rec * 4 * M + 16 * n_tiles
    avg_launch_ms = statistics.mean(per)
    achieved = algo_bytes / (avg_launch_ms / 1e3) / 1e9

    # count-only alert mode (glop_scan_count) on the same input: per-pattern counts, no match list
    count_only = None
    if seg is None and not args.no_extras:
        hist = torch.empty(max(w.patterns.n, 1), dtype=torch.int64, device=dev)
        ctot = torch.empty(1, dtype=torch.int64, device=dev)
        cws = a.count_workspace(dev)
        for _ in range(args.warmup):
            a.count_into(text, hist, ctot, workspace=cws, stream=stream)
        stream.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        csteps = min(args.steps, 500)
        c0.record(stream)
        for _ in range(csteps):
            a.count_into(text, hist, ctot, workspace=cws, stream=stream)
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / csteps
        assert int(ctot.item()) == M, "count-only total %d != scan count %d" % (int(ctot.item()), M)
        count_only = {"value": round(8.0 * N / (cms / 1e3) / 1e9, 3), "unit": "Gbit/s", "ms_per_step": round(cms, 5),
                      "steps": csteps, "gpu_launches_per_step": 3,
                      "note": "glop_scan_count: per-pattern occurrence counts, no match list written"}
        del hist, ctot

    # batches: the same work as plain per-segment glop_scan launches on the same stream
    per_segment = None
    if seg is not None and args.per_segment_steps > 0:
        import ctypes
        L = glop.lib()
        segs = w.seg
        nseg = len(segs) - 1
        per_cnt = torch.zeros(nseg, dtype=torch.int64, device=dev)
        big = int(np.max(np.diff(segs))) if nseg else 0
        ws1 = torch.empty(a.workspace_bytes(big), dtype=torch.uint8, device=dev)
        out1 = torch.empty((max(M, 1), 2), dtype=torch.int32, device=dev)
        tp, op, cp, wp = text.data_ptr(), out1.data_ptr(), per_cnt.data_ptr(), ws1.data_ptr()
        h, sh = a.handle, stream.cuda_stream
        lens = np.diff(segs).astype(np.uint64)
        starts = segs[:-1].astype(np.uint64)

        def per_segment_pass(bases, caps):
            for f in range(nseg):
                rc = L.glop_scan(h, tp + int(starts[f]), int(lens[f]), op + 8 * int(bases[f]), int(caps[f]),
                                 cp + 8 * f, wp, ws1.numel(), sh)
                assert rc == 0, rc
        # first pass: counts only; then every file writes at its place in one output, as the batch does
        per_segment_pass(np.zeros(nseg, np.int64), np.zeros(nseg, np.int64))
        stream.synchronize()
        caps = per_cnt.cpu().numpy()
        bases = np.concatenate([[0], np.cumsum(caps)[:-1]])
        per_segment_pass(bases, caps)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.per_segment_steps):
            per_segment_pass(bases, caps)
        e1.record(stream)
        stream.synchronize()
        wall = (time.perf_counter() - t0) / args.per_segment_steps
        gpu_ms = e0.elapsed_time(e1) / args.per_segment_steps
        assert int(per_cnt.sum().item()) == M
        per_segment = {"launches_per_step": 2 * nseg, "ms_per_step": round(max(gpu_ms, wall * 1e3), 3),
                       "gpu_ms_per_step": round(gpu_ms, 3), "host_ms_per_step": round(wall * 1e3, 3),
                       "value": round(8.0 * N / (max(gpu_ms, wall * 1e3) / 1e3) / 1e9, 3), "unit": "Gbit/s",
                       "note": "plain glop_scan per segment from Python on one stream (counts only kept per file)"}
        del out1, ws1

    # end to end through the C ABI with host buffers (pinned text in, matches out)
    e2e = None
    if seg is None and args.e2e_steps > 0:
        hm = np.empty((M, 2), dtype=np.uint32)
        staging = None
        need = a.workspace_bytes(N)
        import ctypes
        sz = ctypes.c_uint64()
        glop.lib().glop_scan_host_staging_size(a.handle, N, M, ctypes.byref(sz))
        staging = torch.empty(int(sz.value), dtype=torch.uint8, device=dev)
        hm_pinned = torch.empty((M, 2), dtype=torch.int32, pin_memory=True)
        cnt = ctypes.c_uint64()
        hp = host.data_ptr()
        for i in range(2 + args.e2e_steps):
            if i == 2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            rc = glop.lib().glop_scan_host(a.handle, hp, N, hm_pinned.data_ptr(), M, ctypes.byref(cnt),
                                           staging.data_ptr(), staging.numel(), stream.cuda_stream)
            assert rc == 0, rc
        dt = time.perf_counter() - t0
        e2e = {"value": round(8.0 * N * args.e2e_steps * ws / dt / 1e9, 3), "unit": "Gbit/s",
               "h2d_bytes_per_step": N, "d2h_bytes_per_step": 8 + 8 * M}
        if not args.no_extras:
            e2e["link"] = link_roofline(host, staging, hm_pinned, N, M, dt / args.e2e_steps)
        del hm, need

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    line = {
        "metric": "Gbit/s scanned (8*N/t, Eq. 1)", "value": round(gbps, 3), "unit": "Gbit/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_max / args.steps, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "text_bytes": N, "text_sha256": text_sha, "patterns": w.patterns.n,
                   "matches": M,
                   "l2": ("inputs larger than L2 (no flush)" if N > 129e6 else
                          "inputs smaller than L2: a profiling case, not a bench number"),
                   "parallelism": "dp%d (independent shards)" % ws},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": None,
                     "note": "algorithmic bytes = text + halo re-reads + %d B/match + tile status; peak %s"
                             % (rec * 4, which)},
        "clocks": clk,
        "gpu_launches": 2 * args.steps,
        "launch": "cuda graph (memset + init + scan kernel) per step" if plan is not None else "glop_scan per step",
        "verified": verified["ok"], "verification": verified,
        "hbm_input_frac": round(N / (avg_launch_ms / 1e3) / 1e9 / hbm, 4),
        "step_ms": {"mean": round(statistics.mean(per), 5), "median": round(statistics.median(per), 5),
                    "p10": round(float(np.percentile(per, 10)), 5), "p90": round(float(np.percentile(per, 90)), 5),
                    "runs": len(per)},
    }
    if args.smem_budget:
        line["config"]["smem_budget_bytes"] = args.smem_budget
    tr = profiled_traffic(args.workload) if not args.smem_budget else None
    if tr is not None:
        line["roofline"]["traffic"] = tr
    # the limit that binds: instruction issue (4 schedulers per SM, one warp instruction per cycle each)
    ins = profiled_value(args.workload, "issue", "inst_per_launch") if not args.smem_budget else None
    f_sm = (clk or {}).get("sm_mhz") or 2070.0
    if ins is not None:
        peak_issue = 4 * SMS * f_sm * 1e6
        ach = ins / (avg_launch_ms / 1e3)
        line["issue_roofline"] = {"bound": "issue", "achieved": round(ach / 1e12, 4), "peak": round(peak_issue / 1e12, 4),
                                  "unit": "T warp-instructions/s", "frac": round(ach / peak_issue, 4),
                                  "inst_per_launch": ins,
                                  "note": "instructions per launch from the committed ncu summary; peak = 4 x SMs x "
                                          "median SM clock sampled during the timed region"}
    if not args.no_extras:
        rp = read_stream_peak(dev)
        line["roofline"]["read_stream_peak"] = rp
        line["roofline"]["frac_of_read_stream_peak"] = round(achieved / rp, 4)
        ws_stats = walk_stats(w)
        if ws_stats:
            line["walk"] = ws_stats
    if e2e:
        line["e2e"] = e2e
    if count_only:
        line["count_only"] = count_only
    if per_segment:
        line["per_segment_launches"] = per_segment
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    # the metric's other halves on the same box and run: the 20k-signature point and serving
    if args.workload == "syslog-256MiB-1000pat" and not args.no_extras and ws == 1:
        del text, matches, ws_buf, host
        torch.cuda.empty_cache()
        line["dpi_20k"] = dpi_record(dev, args.dpi_steps, args.warmup if args.warmup < 10 else 5, local)
        if args.extra_serve_seconds > 0:
            sv = serve_record(args.extra_serve_seconds, args.serve_hbm_gib, saturated_runs=3)
            sv["note"] = ("the config-5 trace's first %d s of arrivals (200 req/s; the full trace is 60 s: "
                          "bench.py --workload serve)" % args.extra_serve_seconds)
            line["serve"] = sv
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()

"""The native serving loop (glop_server_*): every served request's match list equals the CPU oracle's for its
payload and pattern set -- requests batched across several resident sets in one launch, lone requests on the
idle path, large requests on their own lane -- in real time and saturated."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1704_02278_gb300 import serve  # noqa: E402


def _trace(n, pool_bytes, cap_bytes):
    times, sizes, set_idx = W.config5_requests(200.0, 60.0)
    pools = [torch.from_numpy(W.config5_payload(k, pool_bytes)).pin_memory() for k in (0, 1)]
    reqs = []
    for i in range(n):
        size = int(min(sizes[i], cap_bytes))
        off = (i * 2654435761) % (pool_bytes - size + 1)
        reqs.append(serve.Request(i, int(set_idx[i]), pools[i % 2][off:off + size], float(times[i])))
    return reqs


def _expected(sets, reqs):
    """The oracle once per set, over that set's requests as segments of one buffer."""
    exp = {}
    for si in sorted({r.set_index for r in reqs}):
        rs = [r for r in reqs if r.set_index == si]
        seg = np.zeros(len(rs) + 1, np.uint64)
        seg[1:] = np.cumsum([r.payload.numel() for r in rs])
        buf = np.concatenate([r.payload.numpy() for r in rs]) if seg[-1] else np.zeros(0, np.uint8)
        res = oracle.batch(buf, seg, sets[si].csr())
        cut = np.searchsorted(res[:, 0], np.arange(len(rs) + 1), side="left")
        for k, r in enumerate(rs):
            exp[r.rid] = np.ascontiguousarray(res[cut[k]:cut[k + 1], 1:])
    return exp


def _check(reqs, exp, tag):
    for r in reqs:
        e = exp[r.rid]
        assert r.count == len(e), (tag, r.rid, r.set_index)
        assert np.array_equal(r.matches.reshape(-1, 2), e), (tag, r.rid, r.set_index)
        assert r.done >= 0


def test_native_server_trace_sample_vs_oracle():
    sets = W.config5_sets()
    reqs = _trace(200, 32 << 20, 16 << 20)
    exp = _expected(sets, reqs)
    srv = serve.NativeServer(sets, hbm_budget=2 << 30, keep_matches=True, big_bytes=4 << 20,
                             max_request_bytes=16 << 20)
    try:
        for realtime in (True, False):
            for r in reqs:
                r.count, r.matches, r.done = -1, None, -1.0
            wall, st = srv.serve(reqs, realtime=realtime)
            _check(reqs, exp, realtime)
            assert st["big"] >= 3 and st["batches"] >= 1
            if realtime:
                assert st["fast"] >= 1
                assert all(r.done >= r.arrival for r in reqs)
        assert srv.stats()["sets_per_batch_max"] >= 2  # saturated: one launch over several sets
    finally:
        srv.close()


def test_native_server_empty_tiny_and_tight_budget():
    sets = W.config5_sets()[:3]
    reqs = _trace(40, 4 << 20, 2 << 20)
    empty = torch.empty(0, dtype=torch.uint8).pin_memory()
    for k, r in enumerate(reqs):
        r.set_index %= 3
        if k % 7 == 0:
            r.payload = empty
        elif k % 7 == 1:
            r.payload = r.payload[:3]
    exp = _expected(sets, reqs)
    # a budget of 24 MiB admits a few requests at a time, no lane, no idle path
    srv = serve.NativeServer(sets, hbm_budget=24 << 20, max_inflight=3, keep_matches=True, fast_bytes=0,
                             big_bytes=0)
    try:
        for realtime in (False, True):
            for r in reqs:
                r.count, r.matches, r.done = -1, None, -1.0
            srv.serve(reqs, realtime=realtime)
            _check(reqs, exp, realtime)
        assert srv.stats()["admission_waits"] > 0
    finally:
        srv.close()


def test_native_server_idle_path_rows_and_retries():
    """Lone requests on an idle server with more matches per byte than the server has seen so far: the idle
    path's rows (sized from the set's density so far) overflow, and the request is scanned again with the exact
    count while that fits the idle path, else as a batch; every result still equals the oracle's."""
    sets = [W.Patterns.from_list([b"a", b"aa"]), W.Patterns.from_list([b"ab", b"abab", b"b"])]
    a = np.full(1 << 20, ord("a"), np.uint8)
    ab = np.frombuffer(b"ab" * (1 << 17), np.uint8)
    payloads = [(0, a[:256 << 10]), (1, ab[:100000]), (0, a[:900 << 10]), (0, a[:256 << 10]), (1, ab[:3])]
    reqs = [serve.Request(i, si, torch.from_numpy(p.copy()).pin_memory(), 0.05 * i)
            for i, (si, p) in enumerate(payloads)]
    exp = _expected(sets, reqs)
    srv = serve.NativeServer(sets, hbm_budget=1 << 30, keep_matches=True, fast_bytes=1 << 20, big_bytes=0)
    try:
        wall, st = srv.serve(reqs, realtime=True)
        _check(reqs, exp, "idle")
        assert reqs[0].count == 2 * (256 << 10) - 1
        # the first 256 KiB request overflows its density-sized rows and is scanned again on the idle path;
        # the 900 KiB one has more matches than the idle path holds and becomes a batch
        assert st["rescans"] >= 1 and st["fast"] >= 3 and st["batches"] >= 1
    finally:
        srv.close()

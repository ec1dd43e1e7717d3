"""Serving: every request's result is the same alone and in the continuous-batching mix, and each
equals the CPU oracle's match list for its payload and pattern set."""
import hashlib

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402
from paper_1704_02278_gb300 import serve  # noqa: E402


def _requests(n=80, max_size=2 << 20, span=0.4):
    times, sizes, sets = W.config5_requests()
    pools = [torch.from_numpy(W.config5_payload(k, 8 << 20)).pin_memory() for k in (0, 1)]
    reqs = []
    for i in range(n):
        size = int(min(sizes[i], max_size))
        off = (i * 2654435761) % ((8 << 20) - size + 1)
        reqs.append(serve.Request(i, int(sets[i]), pools[i % 2][off:off + size], times[i] * span / times[n - 1]))
    return reqs


_ORACLE_CACHE = {}


def _oracle(sets, r):
    """The oracle's (offset, pattern_id) list for one request (cached by the contents of its pattern set
    and payload)."""
    pats = sets[r.set_index]
    text = r.payload.numpy()
    key = (hashlib.sha1(pats.buf.tobytes() + pats.offs.tobytes()).hexdigest(), hashlib.sha1(text).hexdigest())
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle.ac_mt(text, pats.csr())
    return _ORACLE_CACHE[key]


def _solo(sets, reqs):
    """Each request scanned alone on the GPU; every solo result must equal the oracle's before it is
    used as the expected value of a served run."""
    autos = {}
    out = []
    for r in reqs:
        a = autos.setdefault(r.set_index, glop.Automaton(sets[r.set_index]))
        if r.payload.numel() == 0:
            out.append(np.zeros((0, 2), np.uint32))
        else:
            m, n = a.scan(r.payload.cuda())
            out.append(m.cpu().numpy().view(np.uint32))
        ref = _oracle(sets, r)
        assert np.array_equal(out[-1].reshape(-1, 2), ref), ("solo scan != oracle", r.rid)
    return out


def test_batched_results_equal_solo_results():
    sets = W.config5_sets()
    reqs = _requests()
    exp = _solo(sets, reqs)
    srv = serve.BatchServer(sets, hbm_budget=1 << 30, keep_matches=True)
    wall, st = srv.serve(reqs, realtime=True)
    assert st["batches"] >= 1 and st["fast"] >= 1  # lone small requests take the idle fast path
    for r, e in zip(reqs, exp):
        assert r.count == len(e), r.rid
        assert np.array_equal(r.matches, e), r.rid


def test_tight_budget_admission_and_saturation():
    sets = W.config5_sets()[:4]
    reqs = _requests(60)
    for r in reqs:
        r.set_index %= 4
    exp = _solo(sets, reqs)
    srv = serve.BatchServer(sets, hbm_budget=40 << 20, max_inflight=3, keep_matches=True)
    wall, st = srv.serve(reqs, realtime=False)
    assert st["admission_waits"] > 0
    for r, e in zip(reqs, exp):
        assert np.array_equal(r.matches, e), r.rid


def test_plain_server_matches():
    sets = W.config5_sets()[:3]
    reqs = _requests(20)
    for r in reqs:
        r.set_index %= 3
    exp = _solo(sets, reqs)
    srv = serve.PlainServer(sets, max_request_bytes=2 << 20, keep_matches=True)
    srv.serve(reqs, realtime=False)
    for r, e in zip(reqs, exp):
        assert np.array_equal(r.matches, e), r.rid


def test_results_larger_than_pinned_buffer_and_rescans():
    sets = W.config5_sets()[:2]
    reqs = _requests(30)
    for r in reqs:
        r.set_index %= 2
    exp = _solo(sets, reqs)
    srv = serve.BatchServer(sets, hbm_budget=1 << 30, keep_matches=True, out_rows=1024)
    srv.density = [1e-6, 1e-6]  # output bounds far too small at first: rescans, then results past the buffer
    wall, st = srv.serve(reqs, realtime=False)
    assert st["rescans"] > 0
    for r, e in zip(reqs, exp):
        assert r.count == len(e), r.rid
        assert np.array_equal(r.matches, e), r.rid


def test_empty_and_tiny_requests():
    sets = W.config5_sets()[:2]
    reqs = _requests(24)
    empty = torch.empty(0, dtype=torch.uint8).pin_memory()
    for k, r in enumerate(reqs):
        r.set_index %= 2
        if k % 5 == 0:
            r.payload = empty
        elif k % 5 == 1:
            r.payload = r.payload[:3]
    exp = _solo(sets, [r for r in reqs])
    for realtime in (True, False):
        srv = serve.BatchServer(sets, hbm_budget=1 << 30, keep_matches=True)
        for r in reqs:
            r.count, r.matches, r.done = -1, None, -1.0
        srv.serve(reqs, realtime=realtime)
        for r, e in zip(reqs, exp):
            assert r.count == len(e), (realtime, r.rid)
            assert np.array_equal(r.matches.reshape(-1, 2), e.reshape(-1, 2)), (realtime, r.rid)


def test_config5_trace_sample_vs_oracle():
    """The first 200 requests of the 60 s, 200 req/s serving trace (all 8 resident sets, the 20,000-pattern
    set included; syslog and packet payloads; trace sizes up to 16 MiB), served by continuous batching at the
    trace's own arrival times and then saturated: every request's match list equals the oracle's."""
    sets = W.config5_sets()
    times, sizes, set_idx = W.config5_requests(200.0, 60.0)
    n = 200
    pool = 32 << 20
    pools = [torch.from_numpy(W.config5_payload(k, pool)).pin_memory() for k in (0, 1)]
    reqs = []
    for i in range(n):
        size = int(min(sizes[i], 16 << 20))
        off = (i * 2654435761) % (pool - size + 1)
        reqs.append(serve.Request(i, int(set_idx[i]), pools[i % 2][off:off + size], float(times[i])))
    assert {r.set_index for r in reqs} == set(range(8))
    assert any(r.set_index == 7 and r.rid % 2 == 1 for r in reqs)  # 20k set on packet payloads
    assert any(r.set_index == 7 and r.rid % 2 == 0 for r in reqs)  # 20k set on syslog payloads
    # the oracle once per set, over that set's requests as segments of one buffer
    exp = {}
    for si in range(8):
        rs = [r for r in reqs if r.set_index == si]
        seg = np.zeros(len(rs) + 1, np.uint64)
        seg[1:] = np.cumsum([r.payload.numel() for r in rs])
        buf = np.concatenate([r.payload.numpy() for r in rs])
        res = oracle.batch(buf, seg, sets[si].csr())
        cut = np.searchsorted(res[:, 0], np.arange(len(rs) + 1), side="left")
        for k, r in enumerate(rs):
            exp[r.rid] = np.ascontiguousarray(res[cut[k]:cut[k + 1], 1:])
    # requests of 4 MiB and more take the large-request lane (end-to-end scans in a worker thread); its result
    # rows are sized far too small at first, so it also grows them and scans again
    srv = serve.BatchServer(sets, hbm_budget=2 << 30, keep_matches=True, big_bytes=4 << 20,
                            max_request_bytes=16 << 20, big_out_rows=1 << 16)
    assert sum(r.payload.numel() >= (4 << 20) for r in reqs) >= 3
    for realtime in (True, False):
        for r in reqs:
            r.count, r.matches, r.done = -1, None, -1.0
        wall, st = srv.serve(reqs, realtime=realtime)
        assert st["batches"] >= 1 and st["big"] >= 3
        if not realtime:  # saturated: one launch carries requests of several resident sets
            assert st["sets_per_batch_max"] >= 2
        assert all(r.done >= r.arrival or not realtime for r in reqs)
        for r in reqs:
            e = exp[r.rid]
            assert r.count == len(e), (realtime, r.rid, r.set_index)
            assert np.array_equal(r.matches.reshape(-1, 2), e), (realtime, r.rid, r.set_index)
    assert srv.big.rescans >= 1
    srv.close()

"""Full-size configurations in the launch configuration the benchmark times.

The DPI and file-batch outputs are far too large for the oracle to redo in
full (the 5,000-pattern file set yields ~1.7 matches per text byte), so these
tests check properties that hold at any size on the whole device output --
sorted, no duplicates, every segment in range -- and compare randomly sampled
segments element by element against the oracle run on just those segments.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def _check_sorted_unique(m, chunk=1 << 26):
    """(segment, offset) non-decreasing and pattern ids strictly increasing within an offset, in chunks."""
    prev = None
    for a in range(0, m.shape[0], chunk):
        b = min(m.shape[0], a + chunk + 1)
        part = m[a:b]
        key = (part[:, 0].to(torch.int64) << 32) | (part[:, 1].to(torch.int64) & 0xFFFFFFFF)
        d = key[1:] - key[:-1]
        assert bool((d >= 0).all()), "not sorted by (segment, offset)"
        pid = part[:, 2].to(torch.int64) & 0xFFFFFFFF
        same = d == 0
        assert bool((pid[1:][same] > pid[:-1][same]).all()), "pattern ids not strictly increasing"
        del key, d, pid, same
    return m[:, 0]


def _sampled(w, m, n, k, rng):
    _check_sorted_unique(m[:n])
    seg_col = m[:n, 0].contiguous()
    nseg = len(w.seg) - 1
    assert int(seg_col[-1]) < nseg
    sel = np.sort(rng.choice(nseg, size=min(k, nseg), replace=False))
    sel_t = torch.tensor(sel, dtype=torch.int32, device=m.device)
    lo = torch.searchsorted(seg_col, sel_t).cpu().numpy()
    hi = torch.searchsorted(seg_col, sel_t + 1).cpu().numpy()
    # one oracle call over the sampled segments, laid end to end
    parts = [w.text[int(w.seg[x]):int(w.seg[x + 1])] for x in sel]
    offs = np.zeros(len(sel) + 1, np.uint64)
    offs[1:] = np.cumsum([len(x) for x in parts])
    exp = oracle.batch(np.concatenate(parts) if parts else np.zeros(0, np.uint8), offs, w.patterns.csr())
    ek = exp[:, 0].astype(np.int64)
    elo = np.searchsorted(ek, np.arange(len(sel)))
    ehi = np.searchsorted(ek, np.arange(len(sel)) + 1)
    checked = 0
    for k, (x, a, b) in enumerate(zip(sel, lo, hi)):
        e = exp[elo[k]:ehi[k]].copy()
        e[:, 0] = x
        got = m[a:b].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, e), x
        checked += len(e)
    return checked


def _run_batch(w):
    a = glop.Automaton(w.patterns)
    d = torch.from_numpy(w.text).cuda()
    s = torch.from_numpy(w.seg.view(np.int64).copy()).cuda()
    m, n = a.scan_batch(d, s)
    return a, m, n


def test_config2_full_size():
    """256 MiB syslog, 1,000 patterns: every match against the multi-threaded oracle."""
    w = W.config2()
    a = glop.Automaton(w.patterns)
    m, n = a.scan(torch.from_numpy(w.text).cuda())
    exp = oracle.ac_mt(w.text, w.patterns.csr())
    assert n == len(exp)
    assert np.array_equal(m.cpu().numpy().view(np.uint32), exp)


def test_config3_full_size_dpi():
    """2 GiB of packets, 20,000 signatures: invariants + 2,000 sampled packets."""
    w = W.config3()
    a, m, n = _run_batch(w)
    assert n > 0
    assert _sampled(w, m, n, 2000, np.random.default_rng(3)) > 0


def test_config4_full_size_files():
    """10,000 log-normal files (~4.1 GB), 5,000 patterns: invariants + 60 sampled files."""
    w = W.config4()
    a, m, n = _run_batch(w)
    assert n > 0
    assert _sampled(w, m, n, 60, np.random.default_rng(4)) > 0

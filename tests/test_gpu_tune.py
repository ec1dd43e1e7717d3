"""Autotuner: every candidate is a valid configuration, and the options it
picks scan bit-exactly."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def test_tune_single_and_cache(tmp_path):
    w = W.config2(4 * W.MiB)
    d = torch.from_numpy(w.text).cuda()
    cache = str(tmp_path / "tune.json")
    r = glop.tune(w.patterns, d, repeats=2, cache_path=cache)
    assert not r["cached"] and len(r["points"]) >= 2
    assert all(pt["gbps"] > 0 for pt in r["points"])
    assert glop.tune(w.patterns, d, repeats=2, cache_path=cache)["cached"]
    a = glop.Automaton(w.patterns, options=r["best"])
    m, n = a.scan(d)
    assert np.array_equal(m.cpu().numpy().view(np.uint32), oracle.ac_mt(w.text, w.patterns.csr()))


def test_tune_batch_dpi_options_exact():
    p = W.config3_patterns()
    seg = W.packet_offsets(W.seed(3, 3), 16 * W.MiB)
    t = W.packets(W.seed(3, 0), W.seed(3, 2), seg, 0.6, 0.01, p)
    d = torch.from_numpy(t).cuda()
    s = torch.from_numpy(seg.view(np.int64).copy()).cuda()
    r = glop.tune(p, d, seg_offsets=s, repeats=1)
    exp = oracle.batch(t, seg, p.csr())
    for opts in [r["best"], {"gram_len": 4, "filter_bits_log2": 13}, {"gram_len": 6, "smem_budget_bytes": 0}]:
        a = glop.Automaton(p, options=opts)
        m, n = a.scan_batch(d, s)
        assert np.array_equal(m.cpu().numpy().view(np.uint32), exp), opts
        a.close()


@pytest.mark.parametrize("subtiles", [1, 2])
def test_chunk_sizes_exact(subtiles):
    """Both staged chunk sizes the tuner searches (31 KiB: one 1 KiB sub-tile per consumer warp; 62 KiB: two)
    give the oracle's match lists: a single buffer with a ragged tail, a prefix-mode scan, packets as
    segments, and count-only totals."""
    w = W.config2(3 * W.MiB + 12345)
    d = torch.from_numpy(w.text).cuda()
    a = glop.Automaton(w.patterns, chunk_subtiles=subtiles)
    m, n = a.scan(d)
    assert np.array_equal(m.cpu().numpy().view(np.uint32), oracle.ac_mt(w.text, w.patterns.csr()))
    hist, tot = a.count(d)
    assert tot == n
    a.close()
    a8 = glop.Automaton(w.patterns, prefix_len=8, chunk_subtiles=subtiles)
    m8, n8 = a8.scan(d)
    assert np.array_equal(m8.cpu().numpy().view(np.uint32), oracle.ac_mt(w.text, w.patterns.csr(), 8))
    a8.close()
    p = W.config3_patterns()
    seg = W.packet_offsets(W.seed(3, 3), 8 * W.MiB)
    t = W.packets(W.seed(3, 0), W.seed(3, 2), seg, 0.6, 0.01, p)
    ab = glop.Automaton(p, chunk_subtiles=subtiles)
    mb, nb = ab.scan_batch(torch.from_numpy(t).cuda(), torch.from_numpy(seg.view(np.int64).copy()).cuda())
    assert np.array_equal(mb.cpu().numpy().view(np.uint32), oracle.batch(t, seg, p.csr()))
    ab.close()

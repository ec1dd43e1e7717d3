"""GPU parity of the batch scan (segments: packets, files) against the oracle."""
import random

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def gpu_batch(pats, text, seg, prefix_len=0):
    a = glop.Automaton(pats, prefix_len=prefix_len)
    d = torch.from_numpy(np.ascontiguousarray(text, dtype=np.uint8).copy()).cuda()
    s = torch.from_numpy(np.ascontiguousarray(seg, dtype=np.uint64).view(np.int64).copy()).cuda()
    m, n = a.scan_batch(d, s)
    out = m.cpu().numpy().view(np.uint32).reshape(-1, 3)
    a.close()
    return out, n


def test_small_segments_random():
    rnd = random.Random(77)
    for it in range(30):
        nseg = rnd.randint(1, 400)
        segs = [bytes(rnd.choice(b"abc") for _ in range(rnd.choice([0, 1, 5, 64, 300, 5000]))) for _ in range(nseg)]
        seg = np.zeros(nseg + 1, np.uint64)
        seg[1:] = np.cumsum([len(x) for x in segs])
        text = b"".join(segs)
        minlen = rnd.choice([1, 4, 8])
        pats = [bytes(rnd.choice(b"abc") for _ in range(rnd.randint(minlen, minlen + 6))) for _ in range(20)]
        exp = oracle.batch(text, seg, pats, method="naive")
        got, n = gpu_batch(pats, np.frombuffer(text, np.uint8), seg)
        assert np.array_equal(got, exp), it


def test_many_empty_segments():
    """More segment boundaries inside one tile than the on-chip list holds."""
    text = b"abcdabcd" * 1000
    cuts = sorted([0, len(text)] + [random.Random(3).randrange(len(text)) for _ in range(3000)])
    seg = np.array(cuts, np.uint64)
    pats = [b"abcd", b"dabc", b"cdab"]
    exp = oracle.batch(text, seg, pats, method="naive")
    got, _ = gpu_batch(pats, np.frombuffer(text, np.uint8), seg)
    assert np.array_equal(got, exp)


def test_segments_not_covering_text():
    text = b"abcdabcdabcd" * 500
    seg = np.array([100, 100, 1000, 3000, 3001], np.uint64)
    pats = [b"abcd", b"bcda"]
    exp = oracle.batch(text, seg, pats, method="naive")
    got, _ = gpu_batch(pats, np.frombuffer(text, np.uint8), seg)
    assert np.array_equal(got, exp)


def test_malformed_offsets_rejected():
    a = glop.Automaton([b"abcd"])
    d = torch.zeros(10000, dtype=torch.uint8, device="cuda")
    s = torch.tensor([0, 5000, 4000, 10000], dtype=torch.int64, device="cuda")
    with pytest.raises(glop.GlopError) as e:
        a.scan_batch(d, s)
    assert e.value.code == glop.EINVAL
    a.close()


def test_dpi_packets_slice():
    p = W.config3_patterns()
    seg = W.packet_offsets(W.seed(3, 3), 64 * W.MiB)
    t = W.packets(W.seed(3, 0), W.seed(3, 2), seg, 0.6, 0.01, p)
    exp = oracle.batch(t, seg, p.csr())
    got, n = gpu_batch(p, t, seg)
    assert n == len(exp) and len(exp) > 0
    assert np.array_equal(got, exp)


def test_files_slice():
    p = W.config4_patterns()
    sizes = W.config4_sizes(300)
    seg = np.zeros(301, np.uint64)
    seg[1:] = np.cumsum(sizes)
    t = W.syslog_files(W.seed(4, 0), W.seed(4, 2), seg, 0.02, p)
    exp = oracle.batch(t, seg, p.csr())
    got, n = gpu_batch(p, t, seg)
    assert np.array_equal(got, exp)


def test_dense_batch_overflow_scratch():
    segs = [b"a" * 5000, b"ab" * 3000, b"a" * 70000, b"", b"ba" * 10]
    seg = np.zeros(len(segs) + 1, np.uint64)
    seg[1:] = np.cumsum([len(x) for x in segs])
    text = b"".join(segs)
    pats = [b"aaaa", b"abab", b"baba", b"aaaaa"]
    exp = oracle.batch(text, seg, pats, method="naive")
    got, _ = gpu_batch(pats, np.frombuffer(text, np.uint8), seg)
    assert np.array_equal(got, exp)



def test_segments_not_covering_the_whole_buffer():
    # bytes before the first segment and after the last one belong to no segment; empty segments anywhere
    rnd = random.Random(5)
    text = bytes(rnd.choice(b"abcab") for _ in range(300_000))
    cuts = sorted(rnd.sample(range(5000, 290_000), 400))
    cuts += [cuts[10], cuts[10], cuts[200]]  # empty segments
    seg = np.array(sorted([3001] + cuts + [290_000, 290_000]), np.uint64)
    pats = [b"abca", b"cab", b"bcabc", b"aaaa", b"b"]
    exp = oracle.batch(text, seg, pats, method="naive")
    got, n = gpu_batch(pats, np.frombuffer(text, np.uint8), seg)
    assert n == len(exp)
    assert np.array_equal(got, exp)

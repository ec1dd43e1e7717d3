"""GPU parity: the CUDA scan through the C ABI against the CPU oracle, bit-exact.

Sizes span many 4 KiB tiles with ragged tails; full-size configurations
compare every match against the multi-threaded Aho-Corasick oracle.
"""
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


def _dev(text: np.ndarray, misalign: int = 0):
    t = np.ascontiguousarray(text, dtype=np.uint8).reshape(-1)
    if misalign == 0:
        return torch.from_numpy(t.copy()).cuda()
    big = torch.zeros(t.size + misalign + 16, dtype=torch.uint8, device="cuda")
    v = big[misalign:misalign + t.size]
    v.copy_(torch.from_numpy(t.copy()))
    return v


def gpu_scan(pats, text, prefix_len=0, misalign=0, capacity=None):
    a = glop.Automaton(pats, prefix_len=prefix_len)
    d = _dev(text, misalign)
    m, n = a.scan(d, capacity=capacity)
    out = m.cpu().numpy().view(np.uint32).reshape(-1, 2)
    a.close()
    return out, n


def _np(b: bytes):
    return np.frombuffer(b, dtype=np.uint8)


def test_worked_example():
    got, n = gpu_scan([b"HIS", b"SHE"], _np(b"SHIS"))
    assert got.tolist() == [[1, 0]]


def test_nested_and_duplicates():
    got, _ = gpu_scan([b"a", b"aa", b"aaa"], _np(b"aaaa"))
    assert got.tolist() == oracle.naive(b"aaaa", [b"a", b"aa", b"aaa"]).tolist()
    pats = [b"abcd", b"abcdef", b"abcd", b"abcdefgh"]
    t = _np(b"xxabcdefghabcdabcdefg")
    assert np.array_equal(gpu_scan(pats, t)[0], oracle.naive(t, pats))


@pytest.mark.parametrize("seed", range(8))
def test_random_small(seed):
    rnd = random.Random(1000 + seed)
    for it in range(40):
        alpha = rnd.choice([b"ab", b"abc", bytes(range(256)), b"a\x00\xff"])
        n = rnd.randint(0, 20000)
        text = bytes(rnd.choice(alpha) for _ in range(n))
        minlen = rnd.choice([1, 2, 4, 5, 8, 12])
        pats = []
        for _ in range(rnd.randint(0, 30)):
            L = rnd.randint(minlen, minlen + 10)
            if text and rnd.random() < 0.7:
                i = rnd.randrange(len(text))
                p = text[i:i + L]
                p = p + bytes(rnd.choice(alpha) for _ in range(L - len(p)))
            else:
                p = bytes(rnd.choice(alpha) for _ in range(L))
            pats.append(p)
        pl = rnd.choice([0, 0, 0, 3, 8])
        exp = oracle.naive(text, pats, pl)
        got, cnt = gpu_scan(pats, _np(text), pl, misalign=rnd.choice([0, 0, 1, 7]))
        assert cnt == len(exp)
        assert np.array_equal(got, exp), (seed, it, len(text), pats[:3], pl)


def test_tile_boundaries():
    """Patterns planted across every 4 KiB tile boundary and at the text end."""
    rnd = random.Random(5)
    n = 4096 * 12 + 777
    t = bytearray(rnd.choice(b"xyz") for _ in range(n))
    pats = [b"straddle-the-tile-boundary", b"tile-b", b"QQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQQ"]
    for k in range(1, 13):
        j = (k * 3) % 26 + 1
        at = k * 4096 - j
        t[at:at + len(pats[0])] = pats[0]
    t[-len(pats[2]):] = pats[2]
    t = bytes(t)
    exp = oracle.naive(t, pats)
    assert (exp[:, 1] == 0).sum() == 12
    got, _ = gpu_scan(pats, _np(t))
    assert np.array_equal(got, exp)


def test_all_byte_values():
    text = np.tile(np.arange(256, dtype=np.uint8), 300)
    pats = [bytes([b, (b + 1) % 256, (b + 2) % 256, (b + 3) % 256]) for b in range(0, 256, 3)]
    pats += [b"\x00\x01\x02\x03\x04\x05\x06\x07\x08", b"\xfe\xff\x00\x01"]
    got, _ = gpu_scan(pats, text)
    assert np.array_equal(got, oracle.ac(text, pats))


def test_empty_cases():
    assert gpu_scan([b"abcd"], np.zeros(0, np.uint8))[1] == 0
    assert gpu_scan([], _np(b"abcdabcd"))[1] == 0
    assert gpu_scan([b"abcd"], _np(b"abc"))[1] == 0


def test_zero_length_pattern_rejected():
    with pytest.raises(glop.GlopError) as e:
        glop.Automaton([b"abcd", b""])
    assert e.value.code == glop.EINVAL


def test_long_patterns_beyond_halo():
    """Patterns longer than the staged halo read the rest of the text from global memory."""
    rnd = random.Random(9)
    base = bytes(rnd.choice(b"ab") for _ in range(3000))
    text = (b"z" * 5000 + base + b"z" * 3000) * 3 + base[:2500]
    pats = [base, base[:1500], base[:2999] + b"b", base[:2999] + b"a", base[100:1200]]
    exp = oracle.naive(text, pats)
    assert len(exp) >= 6
    assert np.array_equal(gpu_scan(pats, _np(text))[0], exp)


def test_overflow_reports_true_count():
    w = W.config1()
    pats = w.patterns
    exp = oracle.ac(w.text, pats.csr())
    a = glop.Automaton(pats)
    d = _dev(w.text)
    cap = len(exp) // 3
    m = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    a.scan_into(d, m, cnt)
    assert a.status(d.device) == glop.EOVERFLOW
    assert int(cnt.item()) == len(exp)
    assert np.array_equal(m.cpu().numpy().view(np.uint32), exp[:cap])
    a.close()


def test_scan_words_count_and_status_in_pinned_memory():
    # glop_scan_words writes the scan's count and status into pinned host words with a kernel
    w = W.config1()
    exp = oracle.ac(w.text, w.patterns.csr())
    a = glop.Automaton(w.patterns)
    L = glop.lib()
    st = torch.cuda.Stream()
    words = torch.zeros(2, dtype=torch.int64, pin_memory=True)
    for cap, status in ((len(exp) + 5, glop.OK), (len(exp) // 3, glop.EOVERFLOW)):
        d = _dev(w.text)
        ws = a.workspace(d.numel(), d.device)
        m = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        words.fill_(-1)
        a.scan_into(d, m, cnt, workspace=ws, stream=st)
        assert L.glop_scan_words(ws.data_ptr(), words.data_ptr(), st.cuda_stream) == glop.OK
        st.synchronize()
        assert words.tolist() == [len(exp), status]
        assert a.status(d.device, stream=st) == status
    # an empty text: count 0, OK
    e = torch.empty(0, dtype=torch.uint8, device="cuda")
    ws = a.workspace(0, e.device)
    a.scan_into(e, None, cnt, workspace=ws, stream=st)
    assert L.glop_scan_words(ws.data_ptr(), words.data_ptr(), st.cuda_stream) == glop.OK
    st.synchronize()
    assert words.tolist() == [0, glop.OK]
    a.close()


def test_config1_full_both_oracles():
    w = W.config1()
    got, n = gpu_scan(w.patterns, w.text)
    assert np.array_equal(got, oracle.naive(w.text, w.patterns.csr()))
    assert np.array_equal(got, oracle.ac(w.text, w.patterns.csr()))


@pytest.mark.parametrize("nbytes", [4096 * 37 + 1, 8 * W.MiB + 12345])
def test_config2_slices(nbytes):
    w = W.config2(nbytes)
    got, n = gpu_scan(w.patterns, w.text)
    assert np.array_equal(got, oracle.ac_mt(w.text, w.patterns.csr()))


def test_prefix_mode_config2_slice():
    w = W.config2(4 * W.MiB)
    got, n = gpu_scan(w.patterns, w.text, prefix_len=8)
    assert np.array_equal(got, oracle.ac_mt(w.text, w.patterns.csr(), 8))


def test_scan_host_matches_device_scan():
    w = W.config2(2 * W.MiB + 3)
    a = glop.Automaton(w.patterns)
    exp = oracle.ac_mt(w.text, w.patterns.csr())
    got, total = a.scan_host(w.text, capacity=len(exp) + 10)
    assert total == len(exp)
    assert np.array_equal(got, exp)
    a.close()


def test_dense_matches_overflow_scratch():
    """Every offset matches: the scratch records overflow and sub-tiles are walked again."""
    text = np.full(1 << 20, ord("a"), np.uint8)
    text[::1000] = ord("b")
    pats = [b"aaaa", b"aaaaaaaa", b"baaa", b"aaaa"]
    got, n = gpu_scan(pats, text)
    exp = oracle.ac_mt(text, pats)
    assert n == len(exp)
    assert np.array_equal(got, exp)


def test_scan_host_pieces_cross_boundaries_and_overflow():
    # long texts are uploaded, scanned and copied back in overlapping pieces; a 199-byte pattern planted
    # across the piece boundaries must be found once, and an overflow keeps the sorted prefix
    w = W.config2(100 * W.MiB + 17)
    longp = bytes(range(1, 200))
    pats = W.Patterns.from_list(w.patterns.as_list() + [longp])
    text = w.text.copy()
    n = text.size
    bounds = glop.host_plan(n)[1:-1]
    assert len(bounds) >= 2
    halo = len(longp) - 1
    for b in bounds:
        # one copy across each piece boundary, and one across the end of the previous piece's look-ahead
        # (rounded up to 4096), where the upload of the next piece begins
        up = (b + halo + 4095) // 4096 * 4096
        text[b - 100:b + 99] = np.frombuffer(longp, np.uint8)
        text[up - 48:up + 151] = np.frombuffer(longp, np.uint8)
    exp = oracle.ac_mt(text, pats.csr())
    a = glop.Automaton(pats)
    pinned = torch.from_numpy(text).pin_memory().numpy()
    got, total = a.scan_host(pinned, capacity=len(exp) + 10)
    assert total == len(exp)
    assert np.array_equal(got, exp)
    long_at = got[got[:, 1] == len(pats.as_list()) - 1][:, 0]
    assert set(b - 100 for b in bounds) | set((b + halo + 4095) // 4096 * 4096 - 48 for b in bounds) <= set(
        int(x) for x in long_at)
    cap = len(exp) // 2 + 7
    got2, total2 = a.scan_host(text, capacity=cap)
    assert total2 == len(exp)
    assert np.array_equal(got2, exp[:cap])
    a.close()


def test_output_lists_past_2_22_entries():
    """More than 2^22 output-list entries in all (here 2^22 + 9 copies of one pattern): a sub-tile's match count
    is summed in 64 bits (the 32-bit sums hold only below that), and one offset expands into millions of rows."""
    n_dup = (1 << 22) + 9
    buf = np.frombuffer(b"ab" * n_dup + b"b", np.uint8).copy()
    offs = np.concatenate([np.arange(0, 2 * n_dup + 1, 2, dtype=np.uint64), np.array([2 * n_dup + 1], np.uint64)])
    pats = W.Patterns(buf, offs)
    text = np.full(3000, ord("x"), np.uint8)
    for i in (0, 7, 2000):  # two "ab" in sub-tile 0, one in sub-tile 1
        text[i:i + 2] = np.frombuffer(b"ab", np.uint8)
    exp = oracle.ac(text, pats.csr())
    assert len(exp) == 3 * (n_dup + 1)
    got, n = gpu_scan(pats, text, capacity=len(exp))
    assert n == len(exp)
    assert np.array_equal(got, exp)

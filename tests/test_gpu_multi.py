"""One batch launch over segments of several automata (glop_scan_batch_multi): each group of segments is
scanned with its own pattern set, and every segment's matches equal the oracle's for that set."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402


def _layout(payloads_per_group):
    """Concatenate each group's payloads, padding every group to a 1 KiB boundary with a segment of its own.
    Returns (text, seg offsets, group starts, [(group, segment) of each payload])."""
    parts, seg, gstart, where = [], [0], [], []
    pos = 0
    for g, pls in enumerate(payloads_per_group):
        gstart.append(pos)
        for p in pls:
            parts.append(p)
            pos += len(p)
            seg.append(pos)
            where.append((g, len(seg) - 2))
        pad = (-pos) % 1024
        if pad:
            parts.append(np.zeros(pad, np.uint8))
            pos += pad
            seg.append(pos)
    gstart.append(pos)
    text = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    return text, np.array(seg, np.uint64), gstart, where


def _run(sets, payloads_per_group, automata=None):
    automata = automata or [glop.Automaton(p) for p in sets]
    text, seg, gstart, where = _layout(payloads_per_group)
    d = torch.from_numpy(text).cuda()
    s = torch.from_numpy(seg.view(np.int64).copy()).cuda()
    ws = torch.empty(automata[0].workspace_bytes(len(text), len(seg) - 1), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cap = max(1024, len(text))
    while True:
        m = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
        glop.scan_batch_multi_into(automata, gstart, d, s, m, cnt, ws)
        st = glop.lib().glop_scan_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream, None)
        n = int(cnt.item())
        if n <= cap:
            assert st == glop.OK, glop.STATUS.get(st)
            break
        cap = n
    got = m[:n].cpu().numpy().view(np.uint32)
    # every payload's segment against the oracle on that payload with its group's set
    for (g, si), p in zip(where, [p for pls in payloads_per_group for p in pls]):
        lo, hi = np.searchsorted(got[:, 0], [si, si + 1])
        exp = oracle.ac(p, sets[g].csr())
        assert np.array_equal(got[lo:hi, 1:], exp), (g, si)
    assert np.all(np.diff(got[:, 0].astype(np.int64)) >= 0)
    return automata


def _payloads(k, sizes, seed):
    rng = np.random.default_rng(seed)
    pool = W.config5_payload(k, 4 << 20)
    out = []
    for sz in sizes:
        o = int(rng.integers(0, len(pool) - sz + 1))
        out.append(pool[o:o + sz].copy())
    return out


def test_multi_groups_of_the_config5_sets():
    sets = W.config5_sets()
    autos = [glop.Automaton(p) for p in sets]
    kinds = [glop.batch_multi_kind(a) for a in autos]
    # the largest group of sets sharing a kernel kind, the 20,000-pattern set included
    kind = kinds[7]
    idx = [i for i, k in enumerate(kinds) if k == kind]
    assert len(idx) >= 3 and 7 in idx
    groups = [[*_payloads(0, [1 + 7 * i, 4096, 70000 + 13 * i], 10 + i), *_payloads(1, [1500, 333], 20 + i)]
              for i in range(len(idx))]
    _run([sets[i] for i in idx], groups, [autos[i] for i in idx])


def test_multi_small_sets_ragged_and_empty_groups():
    sets = W.config5_sets()
    autos = [glop.Automaton(p) for p in sets]
    kinds = [glop.batch_multi_kind(a) for a in autos]
    idx = [i for i, k in enumerate(kinds) if k == kinds[0]]
    # a group with nothing in it, one-byte payloads, payloads that end on and straddle chunk boundaries
    groups = [[], *[_payloads(i % 2, [1, 31 * 1024, 31 * 1024 + 5, 200000], 40 + i) for i in range(len(idx) - 1)]]
    _run([sets[i] for i in idx], groups, [autos[i] for i in idx])
    # the same set twice in one launch, as two groups
    _run([sets[0], sets[0]], [_payloads(0, [5000, 9], 1), _payloads(1, [64, 2048], 2)], [autos[0], autos[0]])


def test_multi_rejects_bad_groups():
    sets = W.config5_sets()
    a = [glop.Automaton(p) for p in sets]
    kinds = [glop.batch_multi_kind(x) for x in a]
    other = next(i for i, k in enumerate(kinds) if k != kinds[0])
    text = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    seg = torch.tensor([0, 1024, 4096], dtype=torch.int64, device="cuda")
    m = torch.empty((64, 3), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(a[0].workspace_bytes(4096, 2), dtype=torch.uint8, device="cuda")
    L = glop.lib()

    def call(autos, gstart):
        hs = (ctypes.c_void_p * len(autos))(*[x.handle.value for x in autos])
        gs = np.ascontiguousarray(gstart, dtype=np.uint64)
        return L.glop_scan_batch_multi(hs, len(autos), gs.ctypes.data, text.data_ptr(), 4096, seg.data_ptr(), 2,
                                       m.data_ptr(), 64, cnt.data_ptr(), ws.data_ptr(), ws.numel(),
                                       torch.cuda.current_stream().cuda_stream)
    assert call([a[0], a[other]], [0, 1024, 4096]) == glop.EINVAL      # two kernel kinds
    assert call([a[0], a[0]], [0, 1000, 4096]) == glop.EINVAL          # a group start off the 1 KiB grid
    assert call([a[0], a[0]], [0, 1024, 4000]) == glop.EINVAL          # the last group does not end the text
    # a group start on the grid that no segment starts at: found on the device
    assert call([a[0], a[0]], [0, 2048, 4096]) == glop.OK
    st = L.glop_scan_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream, None)
    assert st == glop.EINVAL and int(cnt.item()) == 0


def test_multi_short_and_deep_patterns():
    """Several automata of the other kernel kinds in one launch: no start filter (patterns of 1-3 bytes),
    and patterns longer than the staged halo (walks that read past the chunk's staged bytes)."""
    rng = np.random.default_rng(7)
    alpha = np.frombuffer(b"abcd", np.uint8)

    def text(n):
        return alpha[rng.integers(0, 4, n)].copy()

    # no start filter: every set has a pattern shorter than 4 bytes
    short = [W.Patterns.from_list([b"a", b"ab", b"abc", b"dcb", b"abcdabcd"]),
             W.Patterns.from_list([b"b", b"cc", b"dab", b"acbd"])]
    autos = [glop.Automaton(p) for p in short]
    assert glop.batch_multi_kind(autos[0]) == glop.batch_multi_kind(autos[1])
    _run(short, [[text(5000), text(1), text(70000)], [text(31 * 1024), text(3)]], autos)
    # deep: one pattern of 1,500 bytes (longer than the 1 KiB halo) in each set, planted in the payloads
    long_a = text(1500).tobytes()
    long_b = text(1300).tobytes()
    deep = [W.Patterns.from_list([long_a, long_a[:700], b"abca"]), W.Patterns.from_list([long_b, b"dddd", b"cabd"])]
    pa = text(100000)
    pa[31 * 1024 - 600:31 * 1024 - 600 + 1500] = np.frombuffer(long_a, np.uint8)  # across a chunk boundary
    pb = text(70000)
    pb[5000:6300] = np.frombuffer(long_b, np.uint8)
    autos = [glop.Automaton(p) for p in deep]
    assert glop.batch_multi_kind(autos[0]) == glop.batch_multi_kind(autos[1])
    _run(deep, [[pa, text(2000)], [pb]], autos)

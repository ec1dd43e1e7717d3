"""Streaming ingestion, host logic (no GPU): scans of the carried tail plus each chunk, each keeping the
match starts it owns, give exactly the matches of the whole stream."""
import random

import numpy as np

import oracle
from paper_1704_02278_gb300.stream import owned_end


def _streamed(text: bytes, pats, cuts, halo):
    out, buf_start, pos = [], 0, 0
    for k, c in enumerate(cuts):
        pos += c
        final = k == len(cuts) - 1
        b0, b1 = buf_start, pos
        m = oracle.naive(text[b0:b1], pats)
        end = owned_end(b0, b1, halo, final) - b0
        keep = m[m[:, 0] < end].astype(np.int64)
        keep[:, 0] += b0
        out.append(keep)
        buf_start = owned_end(b0, b1, halo, final)
    return np.concatenate(out) if out else np.zeros((0, 2), np.int64)


def test_owned_ranges_tile_the_stream_exactly():
    rnd = random.Random(3)
    for it in range(60):
        alpha = b"ab" if it % 2 else b"abc"
        pats = [bytes(rnd.choice(alpha) for _ in range(rnd.randint(1, 9))) for _ in range(rnd.randint(1, 8))]
        halo = max(len(p) for p in pats) - 1
        text = bytes(rnd.choice(alpha) for _ in range(rnd.randint(0, 400)))
        cuts, left = [], len(text)
        while left:
            c = min(left, rnd.choice([1, 2, halo or 1, 7, 50, 200]))
            cuts.append(c)
            left -= c
        if not cuts:
            cuts = [0]
        got = _streamed(text, pats, cuts, halo)
        exp = oracle.naive(text, pats).astype(np.int64)
        assert np.array_equal(got, exp), (pats, cuts)


def test_owned_end_rules():
    assert owned_end(0, 100, 10, False) == 90
    assert owned_end(95, 100, 10, False) == 95  # a chunk shorter than the halo owns nothing yet
    assert owned_end(95, 100, 10, True) == 100  # the last scan owns everything


def test_native_results_become_views_of_the_rows():
    # glop_ingest hands out (base, pointer to count (offset, pattern_id) rows, count); the wrapper views the rows
    # in place and absolute() adds the base in uint64
    from paper_1704_02278_gb300 import IngestResult
    from paper_1704_02278_gb300.stream import StreamScanner
    rows = np.array([[0, 3], [5, 1], [4294967295, 7]], dtype=np.uint32)
    r = IngestResult(base=(1 << 33) + 11, matches=rows.ctypes.data, count=3)
    res = StreamScanner._result(r)
    assert res.base == (1 << 33) + 11 and len(res) == 3
    assert np.shares_memory(res.matches, rows)
    assert np.array_equal(res.matches, rows)
    assert res.absolute().tolist() == [[(1 << 33) + 11, 3], [(1 << 33) + 16, 1], [(1 << 33) + 11 + 4294967295, 7]]
    empty = StreamScanner._result(IngestResult(base=5, matches=None, count=0))
    assert len(empty) == 0 and empty.absolute().shape == (0, 2)

"""Streaming ingestion on the GPU: chunked scans with the carried halo equal the whole-stream scan."""
import random

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1704_02278_gb300.stream import StreamScanner  # noqa: E402


def _stream(sc, text, cuts, pinned=False):
    parts, pos = [], 0
    for c in cuts:
        chunk = torch.from_numpy(text[pos:pos + c].copy())
        if pinned:
            chunk = chunk.pin_memory()
        parts.append(sc.feed(chunk).absolute())  # (a result's view lives until its slot's next copy-back)
        pos += c
    parts.extend(r.absolute() for r in sc.flush())
    return np.concatenate(parts)


@pytest.mark.parametrize("pinned,depth", [(False, 1), (True, 1), (False, 2), (True, 2), (True, 4)])
def test_config2_stream_in_irregular_chunks(pinned, depth):
    w = W.config2(24 * W.MiB + 321)
    rnd = random.Random(11)
    cuts, left = [], w.text.size
    while left:
        c = min(left, rnd.choice([1, 17, 63, 4096, 1 << 20, 3 << 20, 4 << 20]))
        cuts.append(c)
        left -= c
    sc = StreamScanner(w.patterns, chunk_bytes=4 << 20, out_rows=1 << 20, depth=depth)
    got = _stream(sc, w.text, cuts, pinned)
    exp = oracle.ac_mt(w.text, w.patterns.csr()).astype(np.uint64)
    assert got.shape == exp.shape
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("depth", [1, 2])
def test_small_output_buffer_rescans_and_prefix_mode(depth):
    w = W.config2(6 * W.MiB)
    sc = StreamScanner(w.patterns, chunk_bytes=1 << 20, out_rows=1024, prefix_len=8, depth=depth)
    got = _stream(sc, w.text, [1 << 20] * 6)
    exp = oracle.ac_mt(w.text, w.patterns.csr(), prefix_len=8).astype(np.uint64)
    assert np.array_equal(got, exp)
    assert sc.stats["rescans"] > 0


def test_reset_and_results_held_across_feeds():
    # two streams through one scanner; each result is read after the next feed call, the longest its view
    # is kept
    w = W.config2(5 * W.MiB + 3)
    exp = oracle.ac_mt(w.text, w.patterns.csr()).astype(np.uint64)
    sc = StreamScanner(w.patterns, chunk_bytes=1 << 20, out_rows=1 << 18, depth=2)
    for _ in range(2):
        held, parts = [], []
        for pos in range(0, w.text.size, 1 << 20):
            held.append(sc.feed(torch.from_numpy(w.text[pos:pos + (1 << 20)].copy())))
            if len(held) > 1:
                parts.append(held.pop(0).absolute())
        held.extend(sc.flush())
        parts.extend(r.absolute() for r in held)
        assert np.array_equal(np.concatenate(parts), exp)
        sc.reset()


def test_empty_and_one_byte_chunks():
    w = W.config2(2 * W.MiB + 5)
    cuts, left, k = [], w.text.size, 0
    while left:
        c = min(left, [0, 1, 0, 65536, 1, 300000][k % 6])
        cuts.append(c)
        left -= c
        k += 1
    sc = StreamScanner(w.patterns, chunk_bytes=1 << 20, out_rows=1 << 18, depth=3)
    got = _stream(sc, w.text, cuts)
    exp = oracle.ac_mt(w.text, w.patterns.csr()).astype(np.uint64)
    assert np.array_equal(got, exp)

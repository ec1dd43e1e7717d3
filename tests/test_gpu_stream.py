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
        parts.append(sc.feed(chunk).absolute())  # (a result's view lives until its slot scans again)
        pos += c
    parts.append(sc.flush().absolute())
    return np.concatenate(parts)


@pytest.mark.parametrize("pinned", [False, True])
def test_config2_stream_in_irregular_chunks(pinned):
    w = W.config2(24 * W.MiB + 321)
    rnd = random.Random(11)
    cuts, left = [], w.text.size
    while left:
        c = min(left, rnd.choice([1, 17, 63, 4096, 1 << 20, 3 << 20, 4 << 20]))
        cuts.append(c)
        left -= c
    sc = StreamScanner(w.patterns, chunk_bytes=4 << 20, out_rows=1 << 20)
    got = _stream(sc, w.text, cuts, pinned)
    exp = oracle.ac_mt(w.text, w.patterns.csr()).astype(np.uint64)
    assert got.shape == exp.shape
    assert np.array_equal(got, exp)


def test_small_output_buffer_rescans_and_prefix_mode():
    w = W.config2(6 * W.MiB)
    sc = StreamScanner(w.patterns, chunk_bytes=1 << 20, out_rows=1024, prefix_len=8)
    got = _stream(sc, w.text, [1 << 20] * 6)
    exp = oracle.ac_mt(w.text, w.patterns.csr(), prefix_len=8).astype(np.uint64)
    assert np.array_equal(got, exp)
    assert sc.stats["rescans"] > 0


def test_empty_and_one_byte_chunks():
    w = W.config2(2 * W.MiB + 5)
    cuts, left, k = [], w.text.size, 0
    while left:
        c = min(left, [0, 1, 0, 65536, 1, 300000][k % 6])
        cuts.append(c)
        left -= c
        k += 1
    sc = StreamScanner(w.patterns, chunk_bytes=1 << 20, out_rows=1 << 18)
    got = _stream(sc, w.text, cuts)
    exp = oracle.ac_mt(w.text, w.patterns.csr()).astype(np.uint64)
    assert np.array_equal(got, exp)

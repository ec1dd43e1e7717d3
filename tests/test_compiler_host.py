"""The automaton compiler's tables, walked on the host by the GPU's decision
rules (test-only library), against the oracle."""
import random

import numpy as np
import pytest

import hostcheck
import oracle
import workloads as W


def _single(text, pats, prefix_len=0):
    buf, offs = oracle.pattern_csr(pats)
    t = np.frombuffer(bytes(text), np.uint8) if isinstance(text, (bytes, bytearray)) else text
    got, st = hostcheck.scan(t, [0, len(t)], buf, offs, prefix_len)
    return got[:, 1:], st


def test_worked_example():
    got, st = _single(b"SHIS", [b"HIS", b"SHE"])
    assert got.tolist() == [[1, 0]]
    assert st["gram_len"] == 0  # patterns shorter than 4 bytes: no start filter


@pytest.mark.parametrize("seed", range(6))
def test_random_small(seed):
    rnd = random.Random(seed)
    for it in range(150):
        alpha = rnd.choice([b"ab", b"abc", bytes(range(256)), b"a\x00\xff"])
        text = bytes(rnd.choice(alpha) for _ in range(rnd.randint(0, 200)))
        minlen = rnd.choice([1, 4, 5, 8, 9])
        pats = []
        for _ in range(rnd.randint(0, 10)):
            L = rnd.randint(minlen, minlen + 8)
            if text and rnd.random() < 0.6:
                i = rnd.randrange(len(text))
                p = text[i:i + L]
                p = p + bytes(rnd.choice(alpha) for _ in range(L - len(p)))
            else:
                p = bytes(rnd.choice(alpha) for _ in range(L))
            pats.append(p)
        pl = rnd.choice([0, 0, 0, 3, 8])
        exp = oracle.naive(text, pats, pl)
        got, _ = _single(text, pats, pl)
        assert np.array_equal(got, exp), (text, pats, pl)


def test_config1_full():
    w = W.config1()
    exp = oracle.ac(w.text, w.patterns.csr())
    got, st = _single(w.text, w.patterns.csr())
    assert st["gram_len"] == 4
    assert np.array_equal(got, exp)


def test_config2_slice():
    w = W.config2(4 * W.MiB)
    exp = oracle.ac_mt(w.text, w.patterns.csr())
    got, st = _single(w.text, w.patterns.csr())
    assert np.array_equal(got, exp)
    for pl in (8,):
        assert np.array_equal(_single(w.text, w.patterns.csr(), pl)[0], oracle.ac_mt(w.text, w.patterns.csr(), pl))


def test_config3_slice_segments():
    p = W.config3_patterns()
    seg = W.packet_offsets(W.seed(3, 3), 4 * W.MiB)
    t = W.packets(W.seed(3, 0), W.seed(3, 2), seg, 0.6, 0.01, p)
    exp = oracle.batch(t, seg, p.csr())
    got, st = hostcheck.scan(t, seg, p.buf, p.offs)
    assert st["gram_len"] == 8
    assert len(exp) > 0
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("gram_len,bits", [(4, 13), (5, 16), (8, 19), (6, 0)])
def test_filter_options(gram_len, bits):
    """Every start-filter gram length / bitmap size gives the same exact result."""
    p = W.config3_patterns()
    seg = W.packet_offsets(W.seed(3, 3), 2 * W.MiB)
    t = W.packets(W.seed(3, 0), W.seed(3, 2), seg, 0.6, 0.01, p)
    exp = oracle.batch(t, seg, p.csr())
    got, st = hostcheck.scan(t, seg, p.buf, p.offs, gram_len=gram_len, filter_bits=bits)
    assert st["gram_len"] == gram_len
    assert np.array_equal(got, exp)

"""Pins for the CPU oracle: facts fixed by the paper and by the mathematics.

Each ``pin_*`` takes an :class:`oracle.Oracle` and raises AssertionError when
the oracle disagrees with something other than itself:

* the worked example of Sec. 4 (patterns {HIS, SHE}, text "SHIS"),
* exhaustive brute force on tiny inputs (Python slicing, written separately),
* ``bytes.find`` for single-pattern sets (a library routine), also against the
  Knuth-Morris-Pratt oracle on periodic patterns,
* closed-form counts (nested "a"/"aa"/"aaa"), duplicates, all 256 byte values,
  the end-of-text rule, chunk boundaries of the multi-threaded scan (Sec. 4),
  the empty set, invalid patterns, relabelling, shift invariance, prefix mode
  (Sec. 1 and 5) and segments.

``tests/test_oracle_pins.py`` runs every pin on the real oracle and checks
that builds with planted mistakes fail at least one pin.
"""
import itertools
import random

import numpy as np

import oracle as oracle_mod
from conftest import read_golden


def brute(text: bytes, pats, prefix_len: int = 0):
    """All (i, j) with pattern j (cut to prefix_len if > 0) equal to text[i:i+len]."""
    out = []
    n = len(text)
    for i in range(n):
        for j, p in enumerate(pats):
            if prefix_len:
                p = p[:prefix_len]
            if i + len(p) <= n and text[i:i + len(p)] == p:
                out.append((i, j))
    return out


def as_list(arr):
    return [tuple(int(x) for x in row) for row in arr]


def check_all_ways(o, text: bytes, pats, prefix_len=0, threads=(1, 3, 7)):
    exp = brute(text, pats, prefix_len)
    got_n = as_list(o.naive(text, pats, prefix_len))
    assert got_n == exp, ("naive", text, pats, prefix_len, got_n, exp)
    got_a = as_list(o.ac(text, pats, prefix_len))
    assert got_a == exp, ("ac", text, pats, prefix_len, got_a, exp)
    got_k = as_list(o.kmp(text, pats, prefix_len))
    assert got_k == exp, ("kmp", text, pats, prefix_len, got_k, exp)
    for th in threads:
        got_m = as_list(o.ac_mt(text, pats, prefix_len, threads=th))
        assert got_m == exp, ("ac_mt", th, text, pats, prefix_len, got_m, exp)


def pin_worked_example(o):
    hdr, trace = read_golden("aho_corasick_shis.txt")
    pats = [p.encode() for p in hdr["patterns"].split()]
    text = hdr["text"].encode()
    exp = [tuple(int(x) for x in m.split(":")) for m in hdr["matches"].split()]
    assert as_list(o.naive(text, pats)) == exp
    assert as_list(o.ac(text, pats)) == exp
    assert as_list(o.ac_mt(text, pats, threads=2)) == exp
    for method in ("naive", "ac"):
        assert as_list(o.batch(text, [0, len(text)], pats, method=method)) == [(0,) + m for m in exp]
    got = o.ac_trace(text, pats).splitlines()
    assert got == trace, (got, trace)


ALPHA = [b"a", b"b", b"\x00", b"\xff"]


def _tiny_texts(maxlen=5):
    for L in range(maxlen + 1):
        for tup in itertools.product(ALPHA, repeat=L):
            yield b"".join(tup)


def _tiny_pattern_sets():
    singles = [b"".join(t) for L in (1, 2, 3) for t in itertools.product(ALPHA, repeat=L)]
    sets = [[p] for p in singles]
    rnd = random.Random(1704)
    for _ in range(150):
        k = rnd.randint(2, 3)
        sets.append([rnd.choice(singles) for _ in range(k)])
    return sets


def pin_bruteforce_exhaustive(o):
    """Every text of length <= 5 over {a, b, 0x00, 0xff} against 234 pattern sets."""
    texts = list(_tiny_texts(5))
    seg = np.zeros(len(texts) + 1, dtype=np.uint64)
    seg[1:] = np.cumsum([len(t) for t in texts])
    cat = b"".join(texts)
    for k, pats in enumerate(_tiny_pattern_sets()):
        for prefix_len in ((0, 1, 2) if k % 10 == 0 else (0,)):
            exp = []
            for s, t in enumerate(texts):
                exp.extend((s,) + m for m in brute(t, pats, prefix_len))
            for method in ("naive", "ac"):
                got = as_list(o.batch(cat, seg, pats, prefix_len, method=method, threads=3))
                assert got == exp, (method, pats, prefix_len)


def pin_random_small(o):
    rnd = random.Random(20170407)
    for it in range(300):
        alpha = rnd.choice([b"ab", b"abc", bytes(range(256)), b"a\x00\xff"])
        n = rnd.randint(0, 120)
        text = bytes(rnd.choice(alpha) for _ in range(n))
        pats = []
        for _ in range(rnd.randint(1, 8)):
            if text and rnd.random() < 0.5:
                i = rnd.randrange(len(text))
                pats.append(text[i:i + rnd.randint(1, 6)] or b"a")
            else:
                pats.append(bytes(rnd.choice(alpha) for _ in range(rnd.randint(1, 6))))
        check_all_ways(o, text, pats, prefix_len=rnd.choice([0, 0, 0, 1, 2, 3]))


def pin_single_pattern_find(o):
    """Single-pattern sets: the result is the overlapping ``bytes.find`` sequence."""
    rnd = random.Random(7)
    for it in range(200):
        text = bytes(rnd.choice(b"abab\x00") for _ in range(rnd.randint(0, 300)))
        p = bytes(rnd.choice(b"ab\x00") for _ in range(rnd.randint(1, 4)))
        exp, at = [], text.find(p)
        while at >= 0:
            exp.append((at, 0))
            at = text.find(p, at + 1)
        assert as_list(o.naive(text, [p])) == exp
        assert as_list(o.ac(text, [p])) == exp
        assert as_list(o.ac_mt(text, [p], threads=5)) == exp
        assert as_list(o.kmp(text, [p])) == exp


def pin_periodic_kmp(o):
    """Periodic patterns, where Knuth-Morris-Pratt falls back along borders and occurrences overlap
    (Sec. 2, Sec. 7): every way agrees with brute force and with the overlapping bytes.find sequence."""
    rnd = random.Random(1977)
    pats = [b"aa", b"aba", b"abab", b"aabaab", b"abaabaab", b"aaab", b"babbab"]
    for it in range(60):
        text = bytes(rnd.choice(b"ab") for _ in range(rnd.randint(0, 200)))
        for p in pats:
            exp, at = [], text.find(p)
            while at >= 0:
                exp.append((at, 0))
                at = text.find(p, at + 1)
            assert as_list(o.kmp(text, [p])) == exp, (p, text)
        check_all_ways(o, text, pats, threads=(2,))


def pin_nested(o):
    """'a', 'aa', 'aaa' on 'aaaa': 4 + 3 + 2 = 9 matches, listed in closed form."""
    exp = [(i, j) for i in range(4) for j in range(3) if i + j + 1 <= 4]
    assert len(exp) == 9
    for f in (o.naive, o.ac):
        assert as_list(f(b"aaaa", [b"a", b"aa", b"aaa"])) == exp
    assert as_list(o.ac_mt(b"aaaa", [b"a", b"aa", b"aaa"], threads=4)) == exp
    # n copies of 'a' against 'a'*k for k=1..m: sum_k (n-k+1) matches
    n, m = 257, 40
    got = o.ac(b"a" * n, [b"a" * k for k in range(1, m + 1)])
    assert len(got) == sum(n - k + 1 for k in range(1, m + 1))


def pin_duplicates(o):
    pats = [b"ab", b"b", b"ab", b"ab"]
    exp = [(0, 0), (0, 2), (0, 3), (1, 1), (3, 0), (3, 2), (3, 3), (4, 1)]
    for f in (o.naive, o.ac):
        assert as_list(f(b"abxab", pats)) == exp


def pin_all_byte_values(o):
    text = bytes(range(256)) * 2 + b"\x00\x00\xff"
    pats = [b"\x00", b"\xff\x00", bytes(range(250, 256)), b"\x00\x01\x02", b"\x7f\x80", b"\xff", b"\x00\x00\xff"]
    check_all_ways(o, text, pats)
    assert (0, 0) in as_list(o.ac(text, pats))


def pin_end_of_text(o):
    assert as_list(o.ac(b"xxab", [b"ab"])) == [(2, 0)]
    assert as_list(o.naive(b"xxab", [b"ab"])) == [(2, 0)]
    assert as_list(o.ac(b"xxab", [b"abc"])) == []
    assert as_list(o.naive(b"xxab", [b"abc"])) == []
    assert as_list(o.naive(b"ab", [b"b"])) == [(1, 0)]
    assert as_list(o.ac(b"ab", [b"b"])) == [(1, 0)]


def pin_chunk_boundaries(o):
    """A pattern straddling every chunk boundary of the multi-threaded scan."""
    rnd = random.Random(3)
    p = b"boundary-pattern!"  # 17 bytes
    n, th = 1700, 10
    chunk = (n + th - 1) // th
    text = bytearray(bytes(rnd.choice(b"xyz") for _ in range(n)))
    for c in range(1, th):
        j = c % (len(p) - 1) + 1
        at = c * chunk - j
        text[at:at + len(p)] = p
    text = bytes(text)
    exp = brute(text, [p, b"!", b"by"])
    assert len([m for m in exp if m[1] == 0]) == th - 1
    for t in (th, 3, 16):
        assert as_list(o.ac_mt(text, [p, b"!", b"by"], threads=t)) == exp


def pin_empty_and_invalid(o):
    assert len(o.ac(b"abc", [])) == 0
    assert len(o.naive(b"abc", [])) == 0
    assert len(o.ac(b"", [b"a"])) == 0
    assert len(o.batch(b"", [0, 0, 0], [b"a"])) == 0
    assert len(o.kmp(b"abc", [])) == 0 and len(o.kmp(b"", [b"a"])) == 0
    for f in (o.naive, o.ac, o.ac_mt, o.kmp):
        try:
            f(b"abc", [b"a", b""])
        except oracle_mod.OracleError as e:
            assert e.rc == 1
        else:
            raise AssertionError("zero-length pattern accepted")


def pin_relabel(o):
    rnd = random.Random(11)
    text = bytes(rnd.choice(b"abcd") for _ in range(500))
    pats = [bytes(rnd.choice(b"abcd") for _ in range(rnd.randint(1, 4))) for _ in range(12)]
    base = as_list(o.ac(text, pats))
    perm = list(range(len(pats)))
    rnd.shuffle(perm)
    got = as_list(o.ac(text, [pats[perm[k]] for k in range(len(pats))]))
    inv = {perm[k]: k for k in range(len(pats))}
    assert sorted((i, inv[j]) for i, j in base) == got


def pin_shift(o):
    rnd = random.Random(12)
    text = bytes(rnd.choice(b"abcd") for _ in range(400))
    pats = [bytes(rnd.choice(b"abcd") for _ in range(rnd.randint(1, 5))) for _ in range(10)]
    base = as_list(o.ac(text, pats))
    for k in (1, 5, 64):
        got = as_list(o.ac(b"z" * k + text, pats))
        assert got == [(i + k, j) for i, j in base]


def pin_prefix_mode(o):
    rnd = random.Random(13)
    text = bytes(rnd.choice(b"abc") for _ in range(600))
    pats = [bytes(rnd.choice(b"abc") for _ in range(rnd.randint(1, 12))) for _ in range(20)]
    exact = set(as_list(o.ac(text, pats)))
    for K in (1, 3, 8):
        cut = [p[:K] for p in pats]
        pm = as_list(o.ac(text, pats, prefix_len=K))
        assert pm == as_list(o.ac(text, cut))
        assert pm == as_list(o.naive(text, pats, prefix_len=K))
        assert exact <= set(pm)


def pin_segments(o):
    rnd = random.Random(14)
    segs = [bytes(rnd.choice(b"ab") for _ in range(rnd.randint(0, 30))) for _ in range(40)]
    pats = [b"ab", b"ba", b"aab", b"b", b"abab"]
    seg = np.zeros(len(segs) + 1, dtype=np.uint64)
    seg[1:] = np.cumsum([len(s) for s in segs])
    exp = [(s,) + m for s, t in enumerate(segs) for m in brute(t, pats)]
    for method in ("naive", "ac"):
        for th in (1, 4):
            assert as_list(o.batch(b"".join(segs), seg, pats, method=method, threads=th)) == exp


ALL_PINS = [
    pin_worked_example, pin_bruteforce_exhaustive, pin_random_small, pin_single_pattern_find, pin_periodic_kmp,
    pin_nested,
    pin_duplicates, pin_all_byte_values, pin_end_of_text, pin_chunk_boundaries, pin_empty_and_invalid,
    pin_relabel, pin_shift, pin_prefix_mode, pin_segments,
]

"""Seeded synthetic workloads: shape, determinism and recorded hashes."""
import numpy as np

import workloads as W


def test_config1_shape_and_determinism():
    a, b = W.config1(), W.config1()
    assert a.nbytes == 1 << 20
    assert W.sha256(a.text) == W.sha256(b.text)
    L = a.patterns.lengths()
    assert a.patterns.n == 100 and L.min() >= 4 and L.max() <= 32
    lines = a.text.tobytes().split(b"\n")
    assert all(len(x) > 30 for x in lines[:-1])
    assert lines[0][4:5] == b"-" and lines[0][10:11] == b"T" and lines[0][23:24] == b"Z"


def test_config2_patterns_prefix_fraction():
    p = W.config2_patterns()
    pats = p.as_list()
    L = p.lengths()
    assert p.n == 1000 and L.min() >= 4 and L.max() <= 64
    s = set(pats)
    proper_prefixes = sum(1 for x in pats if any(y != x and y.startswith(x) for y in s))
    assert proper_prefixes >= 100


def test_syslog_planting_count():
    p = W.config2_patterns()
    t = np.empty(1 << 20, np.uint8)
    lib = W._load()
    n = lib.synth_syslog(W.seed(2, 0), W.seed(2, 2), t.ctypes.data, t.size, 0.02, p.buf.ctypes.data,
                         p.offs.ctypes.data, p.n)
    lines = t.tobytes().count(b"\n")
    assert 0.01 * lines < n < 0.03 * lines


def test_packets_shape():
    seg = W.packet_offsets(W.seed(3, 3), 1 << 20)
    sizes = np.diff(seg)
    assert int(seg[-1]) == 1 << 20
    assert set(np.unique(sizes[:-1]).tolist()) <= {64, 576, 1500}
    t1 = W.packets(W.seed(3, 0), W.seed(3, 2), seg, 0.6, 0.01, W.config3_patterns())
    t2 = W.packets(W.seed(3, 0), W.seed(3, 2), seg, 0.6, 0.01, W.config3_patterns())
    assert W.sha256(t1) == W.sha256(t2)
    L = W.config3_patterns().lengths()
    assert L.min() >= 8 and L.max() <= 128


def test_files_independent_of_thread_count():
    sizes = W.config4_sizes(64)
    assert sizes.min() >= 4096 and sizes.max() <= 64 << 20
    seg = np.zeros(65, np.uint64)
    seg[1:] = np.cumsum(sizes)
    lib = W._load()
    p = W.Patterns.from_list([b"abcd"])
    outs = []
    for th in (1, 5):
        buf = np.empty(int(seg[-1]), np.uint8)
        lib.synth_syslog_files(W.seed(4, 0), W.seed(4, 2), buf.ctypes.data, seg.ctypes.data, 64, 0.02,
                               p.buf.ctypes.data, p.offs.ctypes.data, 1, th)
        outs.append(W.sha256(buf))
    assert outs[0] == outs[1]


def test_serve_trace():
    times, sizes, sets = W.config5_requests(200.0, 5.0)
    assert 700 < len(times) < 1300
    assert np.all(np.diff(times) > 0)
    assert sizes.min() >= 1024 and sizes.max() <= 256 << 20
    assert sets.min() >= 0 and sets.max() < 8
    s = W.config5_sets()
    assert [x.n for x in s] == list(W.SERVE_SET_SIZES)

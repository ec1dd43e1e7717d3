"""Seeded synthetic workloads shaped like the paper's experiments.

The paper measured on its own unpublished logs, generated with the Mersenne
Twister (Sec. 6), and random pattern sets (Sec. 6); none are available, so
these generators stand in for them.  This module only draws inputs; it holds
none of the search arithmetic and serves the GPU path, the oracle and the
benchmark alike.

Seeds: ``0x6C6F70 + 1000 * config + stream`` with streams 0 vocabulary /
tokens, 1 patterns, 2 text, 3 sizes.  Every buffer's SHA256 can be recorded
(:func:`sha256`) as the paper recorded its logs' hashes (Sec. 6).

Configurations (sizes are binary):

1. 1 MiB syslog text, 100 patterns of 4..32 bytes (70 % vocabulary phrases,
   30 % random printable).
2. 256 MiB syslog text with 2 % of lines carrying a planted pattern; 1,000
   patterns of 4..64 bytes, 10 % of them prefixes of other patterns.
3. 2 GiB of packets (sizes uniform over {64, 576, 1500} B; 60 % HTTP-like,
   40 % uniform bytes; 1 % carry a planted signature); 20,000 signatures of
   8..128 bytes (half HTTP-token fragments, half mixed printable/binary).
4. 10,000 syslog files, log-normal sizes (median 256 KiB, sigma 0.95,
   clipped to [4 KiB, 64 MiB]); one 5,000-pattern set built as in config 2.
5. Serving: Poisson arrivals at 200/s for 60 s, log-normal request sizes
   (median 256 KiB, sigma 2.0, clipped to [1 KiB, 256 MiB]), 8 resident sets
   of {100, 250, 500, 1k, 2k, 5k, 10k, 20k} patterns of 4..128 bytes.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.cpp")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None
_lock = threading.Lock()

SEED_BASE = 0x6C6F70
KiB = 1 << 10
MiB = 1 << 20
GiB = 1 << 30


def seed(config: int, stream: int) -> int:
    return SEED_BASE + 1000 * config + stream


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u8p, u64p = ctypes.c_void_p, ctypes.c_void_p
        u8pp = ctypes.POINTER(ctypes.c_void_p)
        lib.synth_syslog.restype = ctypes.c_uint64
        lib.synth_syslog.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u8p, ctypes.c_uint64, ctypes.c_double,
                                     u8p, u64p, ctypes.c_uint32]
        lib.synth_syslog_files.restype = ctypes.c_uint64
        lib.synth_syslog_files.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u8p, u64p, ctypes.c_uint32,
                                           ctypes.c_double, u8p, u64p, ctypes.c_uint32, ctypes.c_uint32]
        lib.synth_patterns_syslog.restype = ctypes.c_int
        lib.synth_patterns_syslog.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_double, ctypes.c_double, u8pp, u8pp]
        lib.synth_signatures_dpi.restype = ctypes.c_int
        lib.synth_signatures_dpi.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_double, u8pp, u8pp]
        lib.synth_packet_sizes.restype = ctypes.c_uint64
        lib.synth_packet_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p, ctypes.c_uint64]
        lib.synth_packets_fill.restype = ctypes.c_uint64
        lib.synth_packets_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u8p, u64p, ctypes.c_uint64,
                                           ctypes.c_double, ctypes.c_double, u8p, u64p, ctypes.c_uint32,
                                           ctypes.c_uint32]
        lib.synth_lognormal_sizes.restype = None
        lib.synth_lognormal_sizes.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_uint64, ctypes.c_uint64, u64p]
        lib.synth_random_bytes.restype = None
        lib.synth_random_bytes.argtypes = [ctypes.c_uint64, u8p, ctypes.c_uint64]
        lib.synth_free.restype = None
        lib.synth_free.argtypes = [ctypes.c_void_p]
        _lib = lib
        return lib


def _addr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


@dataclasses.dataclass
class Patterns:
    """A pattern set as CSR: ``buf[offs[j]:offs[j+1]]`` is pattern j."""
    buf: np.ndarray   # uint8
    offs: np.ndarray  # uint64, n+1

    @property
    def n(self) -> int:
        return len(self.offs) - 1

    def __getitem__(self, j: int) -> bytes:
        return self.buf[int(self.offs[j]):int(self.offs[j + 1])].tobytes()

    def as_list(self) -> list[bytes]:
        return [self[j] for j in range(self.n)]

    def lengths(self) -> np.ndarray:
        return np.diff(self.offs).astype(np.int64)

    def csr(self):
        return self.buf, self.offs

    @staticmethod
    def from_list(pats) -> "Patterns":
        pats = [bytes(p) for p in pats]
        offs = np.zeros(len(pats) + 1, dtype=np.uint64)
        if pats:
            offs[1:] = np.cumsum([len(p) for p in pats])
        buf = np.frombuffer(b"".join(pats), dtype=np.uint8).copy() if pats else np.zeros(0, np.uint8)
        return Patterns(buf, offs)


def _take_csr(lib, pb, po, n) -> Patterns:
    offs = np.ctypeslib.as_array(ctypes.cast(po, ctypes.POINTER(ctypes.c_uint64)), shape=(n + 1,)).copy()
    tot = int(offs[-1])
    buf = (np.ctypeslib.as_array(ctypes.cast(pb, ctypes.POINTER(ctypes.c_uint8)), shape=(tot,)).copy()
           if tot else np.zeros(0, np.uint8))
    lib.synth_free(pb)
    lib.synth_free(po)
    return Patterns(buf, offs)


def syslog_patterns(vocab_seed: int, pat_seed: int, n: int, minlen: int, maxlen: int,
                    prefix_frac: float = 0.0, vocab_frac: float = 0.7) -> Patterns:
    lib = _load()
    pb, po = ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib.synth_patterns_syslog(vocab_seed, pat_seed, n, minlen, maxlen, prefix_frac, vocab_frac,
                                   ctypes.byref(pb), ctypes.byref(po))
    if rc:
        raise ValueError("synth_patterns_syslog failed (%d)" % rc)
    return _take_csr(lib, pb, po, n)


def dpi_signatures(tok_seed: int, sig_seed: int, n: int, minlen: int, maxlen: int,
                   http_frac: float = 0.5) -> Patterns:
    lib = _load()
    pb, po = ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib.synth_signatures_dpi(tok_seed, sig_seed, n, minlen, maxlen, http_frac, ctypes.byref(pb),
                                  ctypes.byref(po))
    if rc:
        raise ValueError("synth_signatures_dpi failed (%d)" % rc)
    return _take_csr(lib, pb, po, n)


def syslog_text(vocab_seed: int, text_seed: int, nbytes: int, plant_rate: float = 0.0,
                patterns: Patterns | None = None, out: np.ndarray | None = None) -> np.ndarray:
    lib = _load()
    buf = out if out is not None else np.empty(nbytes, dtype=np.uint8)
    assert buf.dtype == np.uint8 and buf.size >= nbytes and buf.flags["C_CONTIGUOUS"]
    p = patterns or Patterns.from_list([])
    lib.synth_syslog(vocab_seed, text_seed, _addr(buf), nbytes, plant_rate, _addr(p.buf), _addr(p.offs), p.n)
    return buf[:nbytes]


def syslog_files(vocab_seed: int, base_seed: int, seg: np.ndarray, plant_rate: float = 0.0,
                 patterns: Patterns | None = None, out: np.ndarray | None = None) -> np.ndarray:
    lib = _load()
    seg = np.ascontiguousarray(seg, dtype=np.uint64)
    total = int(seg[-1])
    buf = out if out is not None else np.empty(total, dtype=np.uint8)
    p = patterns or Patterns.from_list([])
    lib.synth_syslog_files(vocab_seed, base_seed, _addr(buf), _addr(seg), len(seg) - 1, plant_rate,
                           _addr(p.buf), _addr(p.offs), p.n, _threads())
    return buf[:total]


def packet_offsets(size_seed: int, nbytes: int) -> np.ndarray:
    lib = _load()
    n = lib.synth_packet_sizes(size_seed, nbytes, None, 0)
    seg = np.zeros(n + 1, dtype=np.uint64)
    lib.synth_packet_sizes(size_seed, nbytes, _addr(seg), n + 1)
    return seg


def packets(tok_seed: int, fill_seed: int, seg: np.ndarray, http_frac: float = 0.6, plant_rate: float = 0.0,
            patterns: Patterns | None = None, out: np.ndarray | None = None) -> np.ndarray:
    lib = _load()
    seg = np.ascontiguousarray(seg, dtype=np.uint64)
    total = int(seg[-1])
    buf = out if out is not None else np.empty(total, dtype=np.uint8)
    p = patterns or Patterns.from_list([])
    lib.synth_packets_fill(tok_seed, fill_seed, _addr(buf), _addr(seg), len(seg) - 1, http_frac, plant_rate,
                           _addr(p.buf), _addr(p.offs), p.n, _threads())
    return buf[:total]


def lognormal_sizes(size_seed: int, n: int, median: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(n, dtype=np.uint64)
    lib.synth_lognormal_sizes(size_seed, n, float(median), float(sigma), lo, hi, _addr(out))
    return out


def random_bytes(s: int, n: int) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.uint8)
    lib.synth_random_bytes(s, _addr(out), n)
    return out


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(memoryview(np.ascontiguousarray(a))).hexdigest()


# ---------------------------------------------------------------------------
# The five configurations
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    text: np.ndarray                 # uint8
    patterns: Patterns
    seg: np.ndarray | None = None    # uint64 n+1 segment offsets (batch configs)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nbytes(self) -> int:
        return int(self.text.size)


def config1_patterns() -> Patterns:
    return syslog_patterns(seed(1, 0), seed(1, 1), 100, 4, 32, 0.0, 0.7)


def config1(out: np.ndarray | None = None) -> Workload:
    """1 MiB syslog text, 100 patterns of 4..32 bytes."""
    p = config1_patterns()
    t = syslog_text(seed(1, 0), seed(1, 2), 1 * MiB, 0.0, None, out)
    return Workload("syslog-1MiB-100pat", t, p, None, {"config": 1})


def config2_patterns() -> Patterns:
    return syslog_patterns(seed(2, 0), seed(2, 1), 1000, 4, 64, 0.10, 0.7)


def config2(nbytes: int = 256 * MiB, out: np.ndarray | None = None) -> Workload:
    """256 MiB syslog text, 2 % planted lines, 1,000 patterns of 4..64 bytes (10 % prefixes)."""
    p = config2_patterns()
    t = syslog_text(seed(2, 0), seed(2, 2), nbytes, 0.02, p, out)
    return Workload("syslog-%dMiB-1000pat" % (nbytes // MiB) if nbytes >= MiB else "syslog-%dB-1000pat" % nbytes,
                    t, p, None, {"config": 2})


def config3_patterns() -> Patterns:
    return dpi_signatures(seed(3, 0), seed(3, 1), 20000, 8, 128, 0.5)


def config3(nbytes: int = 2 * GiB, out: np.ndarray | None = None) -> Workload:
    """2 GiB of packets (segments), 20,000 signatures of 8..128 bytes."""
    p = config3_patterns()
    seg = packet_offsets(seed(3, 3), nbytes)
    t = packets(seed(3, 0), seed(3, 2), seg, 0.6, 0.01, p, out)
    return Workload("dpi-%dMiB-20000sig" % (nbytes // MiB), t, p, seg, {"config": 3})


def config4_patterns() -> Patterns:
    return syslog_patterns(seed(4, 0), seed(4, 1), 5000, 4, 64, 0.10, 0.7)


def config4_sizes(nfiles: int = 10000) -> np.ndarray:
    return lognormal_sizes(seed(4, 3), nfiles, 256 * KiB, 0.95, 4 * KiB, 64 * MiB)


def config4(nfiles: int = 10000, out: np.ndarray | None = None) -> Workload:
    """10,000 log-normal syslog files, one 5,000-pattern set."""
    p = config4_patterns()
    sizes = config4_sizes(nfiles)
    seg = np.zeros(nfiles + 1, dtype=np.uint64)
    seg[1:] = np.cumsum(sizes)
    t = syslog_files(seed(4, 0), seed(4, 2), seg, 0.02, p, out)
    return Workload("files-%d-5000pat" % nfiles, t, p, seg, {"config": 4})


SERVE_SET_SIZES = (100, 250, 500, 1000, 2000, 5000, 10000, 20000)


def config5_sets() -> list[Patterns]:
    """8 resident sets, patterns of 4..128 bytes: half syslog-style, half DPI-style."""
    sets = []
    for k, n in enumerate(SERVE_SET_SIZES):
        a = syslog_patterns(seed(5, 0), seed(5, 10 + k), n - n // 2, 4, 128, 0.10, 0.7)
        b = dpi_signatures(seed(5, 1), seed(5, 30 + k), n // 2, 4, 128, 0.5)
        buf = np.concatenate([a.buf, b.buf])
        offs = np.concatenate([a.offs, a.offs[-1] + b.offs[1:]])
        sets.append(Patterns(buf, offs))
    return sets


def config5_requests(rate: float = 200.0, duration: float = 60.0):
    """Poisson arrival times (s), request sizes (bytes) and set indices, from one MT19937 stream."""
    rng = np.random.Generator(np.random.MT19937(seed(5, 3)))
    t, times = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        times.append(t)
    n = len(times)
    sizes = np.clip(np.round(np.exp(np.log(256 * KiB) + 2.0 * rng.standard_normal(n))), 1 * KiB, 256 * MiB)
    sets = rng.integers(0, len(SERVE_SET_SIZES), n)
    return np.array(times), sizes.astype(np.int64), sets.astype(np.int64)


def config5_payload(i: int, size: int, out: np.ndarray | None = None) -> np.ndarray:
    """Request i's payload: even requests syslog text, odd requests DPI-style packets in one buffer."""
    if i % 2 == 0:
        return syslog_text(seed(5, 0), seed(5, 100000 + i), size, 0.02, None, out)
    seg = np.array([0, size], dtype=np.uint64)
    return packets(seed(5, 1), seed(5, 100000 + i), seg, 0.6, 0.0, None, out)

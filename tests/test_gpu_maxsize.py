"""The largest single buffer the ABI takes (2^32 - 1 bytes: offsets are 32-bit), and one byte more.

The text tiles a random block in which no pattern occurs, with patterns planted at the start, around
2^31 (offsets with the top bit set), across a 512 MiB piece boundary of the end-to-end path and ending on
the last byte; the expected matches are exactly the planted ones."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1704_02278_gb300 as glop  # noqa: E402

N = (1 << 32) - 1


def _case():
    rng = np.random.default_rng(2024)
    pats = [bytes(rng.integers(0, 256, size=n, dtype=np.uint8)) for n in (9, 12, 16, 31)]
    block = rng.integers(0, 256, size=1 << 20, dtype=np.uint8)
    # no pattern occurs in the block, nor across the seam of two blocks
    assert len(oracle.naive(np.concatenate([block, block[:64]]).tobytes(), pats)) == 0
    text = np.empty(N + 1, np.uint8)  # one spare byte: the 2^32-byte view for the limit check
    text[:] = np.resize(block, N + 1)
    # (no two plants overlap; 512 MiB is a piece boundary of the end-to-end path)
    where = [(0, 0), ((1 << 31) - 20, 2), (1 << 31, 1), ((512 << 20) - 10, 3), ((512 << 20) + 40, 0),
             (3 * (1 << 30) + 12345, 2), (N - 71, 3), (N - 16, 2)]
    for off, j in where:
        text[off:off + len(pats[j])] = np.frombuffer(pats[j], np.uint8)
    # expected: the oracle on a window around every plant (the block itself holds no match)
    found = set()
    for off, j in where:
        lo = max(0, off - 64)
        hi = min(N, off + len(pats[j]) + 64)
        for o, pid in oracle.naive(text[lo:hi].tobytes(), pats):
            found.add((lo + int(o), int(pid)))
    assert {(off, j) for off, j in where} <= found
    exp = np.array(sorted(found), np.uint32)
    return pats, text, exp


@pytest.fixture(scope="module")
def case():
    return _case()


def test_device_scan_at_the_offset_limit(case):
    pats, text, exp = case
    a = glop.Automaton(pats)
    d = torch.from_numpy(text).cuda()
    m, n = a.scan(d[:N], capacity=64)
    assert n == len(exp)
    assert np.array_equal(m.cpu().numpy().view(np.uint32), exp)
    hist, total = a.count(d[:N])
    assert total == len(exp)
    assert hist.cpu().numpy().tolist() == np.bincount(exp[:, 1], minlength=len(pats)).tolist()
    # one byte more than a 32-bit offset can reach is rejected before any launch
    out = torch.empty((16, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    small_ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(glop.GlopError) as e:
        a.scan_into(d, out, cnt, workspace=small_ws)
    assert e.value.code == glop.EINVAL
    a.close()


def test_end_to_end_pieces_at_the_offset_limit(case):
    pats, text, exp = case
    a = glop.Automaton(pats)
    got, total = a.scan_host(text[:N], capacity=64)
    assert total == len(exp)
    assert np.array_equal(got, exp)
    a.close()

"""The piece plan of glop_scan_host (host logic, no GPU): the pieces tile the text, inner bounds are
4096-aligned, full pieces are equal and bounded in number, the first piece is short."""
import ctypes

import pytest

import paper_1704_02278_gb300 as glop
from paper_1704_02278_gb300 import _build

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build_lib()


@pytest.mark.parametrize("n", [0, 1, 4095, 16 * MiB - 1])
def test_short_texts_go_in_one_piece(n):
    assert glop.host_plan(n) == [0, n]


@pytest.mark.parametrize("n", [16 * MiB, 16 * MiB + 1, 20 * MiB + 3, 64 * MiB, 100 * MiB + 17, 256 * MiB, (1 << 30) + 5,
                               (1 << 32) - 1])
def test_long_texts_tile_in_aligned_pieces(n):
    b = glop.host_plan(n)
    assert b[0] == 0 and b[-1] == n
    sizes = [y - x for x, y in zip(b, b[1:])]
    assert all(s > 0 for s in sizes)
    assert all(x % 4096 == 0 for x in b[1:-1])
    assert 3 <= len(sizes) <= 9
    full = sizes[1:]
    assert len(full) <= min(8, n // (8 * MiB))
    assert len(set(full[:-1])) == 1 and full[-1] <= full[0]  # equal, the last one takes what is left
    assert full[-1] > full[0] // 2
    assert full[0] // 5 <= sizes[0] < full[0]


def test_plan_argument_errors():
    lib = glop.lib()
    n = ctypes.c_uint32(99)
    assert lib.glop_scan_host_plan(256 * MiB, None, 0, None) == glop.EINVAL
    small = (ctypes.c_uint64 * 3)()
    assert lib.glop_scan_host_plan(256 * MiB, small, 3, ctypes.byref(n)) == glop.EINVAL
    assert n.value == 9  # the count is set even when the array is too small
    assert lib.glop_scan_host_plan(256 * MiB, None, 0, ctypes.byref(n)) == glop.OK and n.value == 9

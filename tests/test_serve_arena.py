"""Host logic of the serving layer that needs no GPU: the HBM-budget arena."""
import random

import pytest

from paper_1704_02278_gb300.serve import DeviceArena


class _FakeTorch:
    pass


def make_arena(budget):
    a = DeviceArena.__new__(DeviceArena)
    a.size = budget
    a.base = 0
    a.free = [(0, budget)]
    return a


def test_alloc_release_merges_back_to_one_range():
    a = make_arena(1 << 20)
    rnd = random.Random(5)
    live = []
    for it in range(2000):
        if live and (rnd.random() < 0.45 or a.largest_free < 4096):
            o, n = live.pop(rnd.randrange(len(live)))
            a.release(o, n)
        else:
            got = a.alloc(rnd.randint(1, 20000))
            if got:
                o, n = got
                assert o % DeviceArena.ALIGN == 0 and n % DeviceArena.ALIGN == 0
                for o2, n2 in live:
                    assert o + n <= o2 or o2 + n2 <= o, "overlap"
                live.append(got)
    for o, n in live:
        a.release(o, n)
    assert a.free == [(0, 1 << 20)]


def test_alloc_fails_beyond_budget():
    a = make_arena(4096)
    assert a.alloc(4097) is None
    assert a.alloc(4096) == (0, 4096)
    assert a.alloc(1) is None

"""The oracle against the paper's worked example, brute force, library
routines and invariants; and the pins against planted mistakes."""
import pytest

import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=[p.__name__ for p in P.ALL_PINS])
def test_pin(pin):
    pin(oracle.default())


# Each planted mistake of glop_oracle.c (ORACLE_MUTANT=k):
#  1 drops matches that end exactly at the end of the text
#  2 drops the merge output(s) = own(s) U output(fail(s))
#  3 converts end to start position off by one
#  4 overlaps multi-threaded chunks by one byte too few
#  5 removes the failure function (every failure goes to the initial state)
#  6 cuts patterns to prefix_len + 1 bytes in prefix mode
#  7 compares one byte too few in the naive scan
#  8 lets a segment's scan run one byte into the next segment
#  9 restarts Knuth-Morris-Pratt from scratch after an occurrence (drops overlapping ones)
MUTANTS = [1, 2, 3, 4, 5, 6, 7, 8, 9]


@pytest.mark.parametrize("k", MUTANTS)
def test_pins_catch_planted_mistake(k, tmp_path):
    bad = oracle.mutant(k, str(tmp_path))
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(bad)
        except (AssertionError, oracle.OracleError):
            failed.append(pin.__name__)
    assert failed, "planted mistake %d passed every pin" % k

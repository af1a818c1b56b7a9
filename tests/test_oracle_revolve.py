"""Pins of the checkpointing oracle (oracle/revolve.py).

min_advances is a recursion over the first stored state; it is held to
(1) an exhaustive search over all schedules of unit moves on tiny cases and
(2) Griewank's closed form for binomial checkpointing (Griewank 1992,
Griewank & Walther 2000): with S = s + 1 stored states and r the least
integer with C(S + r, r) >= l, the fewest advanced steps are
r l - C(S + r, r - 1).
"""
from math import comb

import pytest

from oracle.revolve import exhaustive_min_advances, min_advances


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_recursion_matches_exhaustive_search(s):
    for l in range(1, 8):
        assert min_advances(l, s) == exhaustive_min_advances(l, s), (l, s)


def _closed_form(l, s):
    S = s + 1
    r = 0
    while comb(S + r, r) < l:
        r += 1
    return 0 if r == 0 else r * l - comb(S + r, r - 1)


def test_recursion_matches_griewank_closed_form():
    for s in range(0, 9):
        for l in range(1, 151):
            assert min_advances(l, s) == _closed_form(l, s), (l, s)


def test_special_cases():
    assert min_advances(1, 0) == 0
    assert min_advances(10, 0) == 45            # every step from step 0 anew
    assert min_advances(10, 9) == 9             # every state stored once
    assert min_advances(1000, 20) == _closed_form(1000, 20)

"""The library's binomial checkpointing schedule (host code, no GPU).

mmod_revolve_schedule is simulated action by action: every step must be
reversed once, in the order nt-1, ..., 0, each with the working state at that
step; a restore must load the state its slot holds; no more slots than
allowed may be used; and the advanced steps must equal the oracle's minimum.
"""
import numpy as np
import pytest

import paper_2007_06048_gb300 as M
from oracle.revolve import min_advances


def simulate(nt, snaps, acts):
    nslots = max(0, min(snaps, nt - 1))
    w, nxt, adv = 0, nt - 1, 0
    slots = {}
    for kind, a, b in acts:
        if kind == M.REV_ADVANCE:
            assert w == a and b > a
            adv += b - a
            w = b
        elif kind == M.REV_SAVE:
            assert 0 <= a < nslots and w == b
            slots[a] = b
        elif kind == M.REV_RESTORE:
            if a == -1:
                assert b == 0
            else:
                assert slots.get(a) == b
            w = b
        elif kind == M.REV_REVERSE:
            assert a == nxt and w == a
            nxt -= 1
        else:
            raise AssertionError(f"unknown action {kind}")
    assert nxt == -1
    return adv


@pytest.mark.parametrize("snaps", [0, 1, 2, 3, 5, 8, 20])
def test_schedule_is_valid_and_optimal(snaps):
    for nt in list(range(1, 40)) + [64, 100, 257]:
        acts, adv = M.mmod_revolve_schedule(nt, snaps)
        assert simulate(nt, snaps, acts) == adv
        assert adv == min_advances(nt, min(snaps, max(nt - 1, 0))), (nt, snaps)


def test_schedule_large():
    acts, adv = M.mmod_revolve_schedule(1000, 20)
    assert simulate(1000, 20, acts) == adv == min_advances(1000, 20)
    assert adv < 3 * 1000   # three sweeps suffice: C(23, 2) >= 1000 with S = 21
    acts, adv = M.mmod_revolve_schedule(5000, 3)
    assert simulate(5000, 3, acts) == adv


def test_schedule_edge_cases():
    acts, adv = M.mmod_revolve_schedule(0, 4)
    assert len(acts) == 0 and adv == 0
    acts, adv = M.mmod_revolve_schedule(7, 100)   # more slots than steps: store every state
    assert adv == 6 and simulate(7, 100, acts) == 6
    lib = M.load()
    assert lib.mmod_revolve_schedule(-1, 2, None, 0, None, None) == -1
    buf = np.zeros((2, 3), np.int32)
    assert lib.mmod_revolve_schedule(30, 2, buf.ctypes.data, 2, None, None) == -1   # cap too small

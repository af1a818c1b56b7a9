"""Checkpointing oracle: the fewest forward steps a reversal needs.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Reversing l time steps means running the adjoint of step l-1, then l-2, ...,
then 0, where the adjoint of step n needs the forward state at step n.  The
state at step 0 is always at hand; besides it, s slots may hold one state
each.  A forward step from the state at n gives the state at n+1.

``min_advances(l, s)`` is the least number of forward steps (not counting the
one forward step each reversal takes from step n itself) over every schedule
that splits the range at the first stored state: take j steps, store the
state there, reverse the last l-j steps with one slot fewer, then the first j
steps with all s slots (the stored state is released):

    T(l, s) = min_{0 < j < l} [ j + T(l - j, s - 1) + T(j, s) ],
    T(1, s) = 0,   T(l, 0) = l (l - 1) / 2   (each step from step 0 anew).

This is plain dynamic programming over the split, evaluated by brute force.
Pins: ``exhaustive_min_advances`` searches all schedules of single-step moves
on tiny cases (no splitting assumption), and the closed form of Griewank
(1992), T = r l - C(s + 1 + r, r - 1) with r the least integer such that
C(s + 1 + r, r) >= l, holds it at larger sizes.
"""
from __future__ import annotations

import heapq
from functools import lru_cache


def min_advances(l: int, s: int) -> int:
    """Least forward steps to reverse l steps with s free slots (brute-force DP)."""
    if l < 0 or s < 0:
        raise ValueError("l and s must be >= 0")

    @lru_cache(maxsize=None)
    def T(n: int, k: int) -> int:
        if n <= 1:
            return 0
        if k == 0:
            return n * (n - 1) // 2
        return min(j + T(n - j, k - 1) + T(j, k) for j in range(1, n))

    # fill the table bottom-up so deep recursion is never needed
    for k in range(s + 1):
        for n in range(l + 1):
            T(n, k)
    return T(l, s)


def exhaustive_min_advances(l: int, s: int) -> int:
    """Dijkstra over all schedules of unit moves (tiny l, s only).

    State: (working step w, frozenset of stored steps, next step to reverse).
    Moves: advance w -> w + 1 (cost 1); store w (if a slot is free); drop a
    stored step; load a stored step or step 0 into w; reverse step `next`
    when w == next (then next - 1).  Done when every step is reversed.
    """
    start = (0, frozenset(), l - 1)
    dist = {start: 0}
    heap = [(0, start)]
    while heap:
        d, st = heapq.heappop(heap)
        if d != dist.get(st):
            continue
        w, stored, nxt = st
        if nxt < 0:
            return d
        moves = []
        if w < nxt:
            moves.append(((w + 1, stored, nxt), 1))
        if w == nxt:
            moves.append(((w, stored, nxt - 1), 0))
        if len(stored) < s and w not in stored and w != 0:
            moves.append(((w, stored | {w}, nxt), 0))
        for q in stored:
            moves.append(((w, stored - {q}, nxt), 0))
            if q != w:
                moves.append(((q, stored, nxt), 0))
        if w != 0:
            moves.append(((0, stored, nxt), 0))
        for ns, c in moves:
            nd = d + c
            if nd < dist.get(ns, 1 << 60):
                dist[ns] = nd
                heapq.heappush(heap, (nd, ns))
    raise RuntimeError("no schedule found")

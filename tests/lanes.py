"""Brute-force per-lane definitions of the warp functions, for tiny grids.

Written from the public PTX definitions of ``shfl.sync``, ``vote.sync`` and
``match.sync`` in element-index form: element i belongs to global thread i,
which is lane ``i % 32`` of its warp and rank ``i % W`` of its width-W tile
(W divides 32, so a tile never straddles two warps).  Plain Python loops over
lists, no numpy vectorisation and nothing shared with the oracle's executor,
so that the two can pin each other.
"""
from __future__ import annotations

SHFL_IDX, SHFL_UP, SHFL_DOWN, SHFL_XOR, BALLOT, ANY, ALL, MATCH_ANY = range(8)


def shfl(fn, x, W, param):
    """Per-lane result of a shuffle; a padding source (index >= n) reads 0."""
    n = len(x)
    out = []
    for i in range(n):
        lane = i % 32
        rank = i % W
        tile0 = i - rank           # first element of i's tile
        warp0 = i - lane           # first element of i's warp
        if fn == SHFL_IDX:
            src = tile0 + (param % W)          # srcLane modulo the width
        elif fn == SHFL_UP:
            src = i - param if rank - param >= 0 else i
        elif fn == SHFL_DOWN:
            src = i + param if rank + param <= W - 1 else i
        else:  # xor: any lane of the warp up to the end of the caller's tile
            j = lane ^ param
            src = warp0 + j if j <= (lane - rank) + W - 1 else i
        out.append(x[src] if src < n else 0)
    return out


def ballot(pred, W):
    """Tile-local ballot: bit r set iff element tile0 + r exists and is true."""
    n = len(pred)
    out = []
    for i in range(n):
        tile0 = i - i % W
        m = 0
        for r in range(W):
            if tile0 + r < n and pred[tile0 + r]:
                m |= 1 << r
        out.append(m)
    return out


def any_all(pred, W, want_all):
    full = (1 << W) - 1
    return [int(m == full) if want_all else int(m != 0) for m in ballot(pred, W)]


def match_any(x, W):
    """Tile-local mask of existing elements equal to the caller's."""
    n = len(x)
    out = []
    for i in range(n):
        tile0 = i - i % W
        m = 0
        for r in range(W):
            if tile0 + r < n and x[tile0 + r] == x[i]:
                m |= 1 << r
        out.append(m)
    return out

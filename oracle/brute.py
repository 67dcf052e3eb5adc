"""Brute-force answers over Python sets, for tiny inputs only.

TEST INFRASTRUCTURE ONLY.

- ``exact_msmt``: the MSMT answer itself (Sec. 1): the IDs i with every term of
  Q in S_i.  RAMBO must return a superset of it (no false negatives, Sec. 4.1).
- ``exact_cell_rambo``: RAMBO with every cell an exact set union instead of a
  Bloom filter (Sec. 3: a cell holds the union of the sets the partition sends
  to it; Algorithm 2 takes, per table, the union of the hit cells' set IDs and
  intersects across tables).  When the Bloom filters have no false positives,
  Algorithm 2 returns exactly this.
"""
from __future__ import annotations


def exact_msmt(sets: dict[int, set[int]], Q) -> list[int]:
    Q = list(Q)
    return sorted(i for i, S in sets.items() if all(x in S for x in Q))


def exact_cell_rambo(sets: dict[int, set[int]], phi, R: int, Q) -> list[int]:
    """phi(r, i) -> cell of set i in table r.  ``sets`` holds the inserted
    (registered) sets; a set with no terms still takes part."""
    Q = list(Q)
    unions: dict[tuple[int, int], set[int]] = {}
    for i, S in sets.items():
        for r in range(R):
            unions.setdefault((r, phi(r, i)), set()).update(S)
    out = []
    for i in sets:
        if all(all(x in unions[(r, phi(r, i))] for x in Q) for r in range(R)):
            out.append(i)
    return sorted(out)

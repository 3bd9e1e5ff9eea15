"""Exact permanents of 0/1 matrices with few zeros, by rook numbers.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

For a board B -- a set of cells (i, j) of the n x n grid -- let J - B be the 0/1
matrix whose zeros are exactly the cells of B.  A permutation contributes 1 to
per(J - B) (Eq. (1), Section 3.1) iff it uses no cell of B.  Inclusion-exclusion
over the cells of B that a permutation does use (Riordan, *An Introduction to
Combinatorial Analysis*, 1958, ch. 7-8) gives

    per(J - B) = sum_{k >= 0} (-1)^k r_k(B) (n - k)!,

where r_k(B) is the number of ways to place k non-attacking rooks on B (k cells
of B, no two in one row or one column): each such placement fixes k values of
the permutation and leaves (n - k)! completions.

This identity uses neither Ryser's formula nor the Store-zechin development, and
Python integers make it exact at any size, so it yields reference values for
dense 0/1 matrices of order 35..40 (permanents far above 2^128) in time
exponential only in |B|.
"""
from __future__ import annotations

import math
from typing import Iterable, List, Sequence, Tuple

Cell = Tuple[int, int]


def rook_numbers(cells: Iterable[Cell]) -> List[int]:
    """r_0, r_1, ... r_|B| of the board `cells` (every non-attacking subset, counted
    once by a depth-first walk over the cells in increasing order)."""
    cs = sorted(set((int(i), int(j)) for i, j in cells))
    r = [0] * (len(cs) + 1)

    def walk(start: int, rows: frozenset, cols: frozenset, k: int) -> None:
        r[k] += 1
        for t in range(start, len(cs)):
            i, j = cs[t]
            if i not in rows and j not in cols:
                walk(t + 1, rows | {i}, cols | {j}, k + 1)

    walk(0, frozenset(), frozenset(), 0)
    return r


def per_complement(n: int, cells: Sequence[Cell]) -> int:
    """per(J_n - B) for the board B = `cells` (0-based cells inside n x n)."""
    for i, j in cells:
        if not (0 <= i < n and 0 <= j < n):
            raise ValueError(f"cell {(i, j)} outside the {n} x {n} grid")
    r = rook_numbers(cells)
    return sum((-1) ** k * rk * math.factorial(n - k) for k, rk in enumerate(r) if k <= n)


def complement_matrix(n: int, cells: Sequence[Cell]):
    """The 0/1 matrix J_n - B as int64 (numpy)."""
    import numpy as np
    a = np.ones((n, n), dtype=np.int64)
    for i, j in cells:
        a[i, j] = 0
    return a

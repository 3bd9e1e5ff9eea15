"""Instrumented Store-zechin (Su & Zheng, arXiv:1802.02779, Section 4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper develops per(A) along the last row (Section 4), then develops each
minor along its own last row, down to small minors, and stores every distinct
sub-permanent the first time it is computed so that later references reuse it
("like zechins").  Property (4) of Section 3.1 (Laplace development without
signs) is the only identity used:

    per(rows 0..r, columns C) = sum_{j in C} a[r, j] * per(rows 0..r-1, C minus j).

This module follows those steps literally with a dictionary of stored
sub-permanents keyed by (last row, column set), in exact Python arithmetic, and
counts the multiplications and additions it performs.  A k x k sub-permanent
(k >= 2) costs k multiplications and k-1 additions the first time it is needed
and nothing afterwards; a 1 x 1 sub-permanent is a matrix entry and costs
nothing.  Counts are attributed to the paper's "Term j" (the j-th product
a[n-1, j] * per(A_{n; j}) of the top development, columns in ascending order)
plus the final sum of the n terms (the paper's row "Sigma"), which is how
Tables 1-3 of Section 4 present them.
"""
from __future__ import annotations

from collections import Counter
from typing import Dict, FrozenSet, List, Tuple

Key = Tuple[int, FrozenSet[int]]


class _Counter:
    def __init__(self):
        self.mul = 0
        self.add = 0


def _develop(a, r: int, cols: FrozenSet[int], store: Dict[Key, object], cnt: _Counter):
    """per(rows 0..r, cols), developing along row r; stores every result."""
    key = (r, cols)
    if key in store:
        return store[key]
    if r == 0:
        (j,) = tuple(cols)
        val = a[0][j]
    else:
        val = None
        for j in sorted(cols):
            sub = _develop(a, r - 1, cols - {j}, store, cnt)
            term = a[r][j] * sub
            cnt.mul += 1
            if val is None:
                val = term
            else:
                val = val + term
                cnt.add += 1
    store[key] = val
    return val


def store_zechin(a):
    """Evaluate per(A) by Store-zechin and count its arithmetic.

    ``a`` is a square nested sequence (or array) of Python numbers.  Returns
    ``(value, table)`` where ``table`` is a dict with keys ``terms`` (list of
    (mul, add) per top-level term j = 0..n-1), ``sigma_add`` (additions of the
    final sum), ``total`` ((mul, add)) and ``stored`` (number of distinct stored
    sub-permanents of order >= 2, the minors themselves excluded).
    """
    a = [list(row) for row in a]
    n = len(a)
    if n == 0:
        return 1, {"terms": [], "sigma_add": 0, "total": (0, 0), "stored": 0}
    if n == 1:
        return a[0][0], {"terms": [(0, 0)], "sigma_add": 0, "total": (0, 0), "stored": 0}
    store: Dict[Key, object] = {}
    terms: List[Tuple[int, int]] = []
    total_val = None
    all_cols = frozenset(range(n))
    for j in range(n):                       # Term j of the top development
        cnt = _Counter()
        minor = _develop(a, n - 2, all_cols - {j}, store, cnt)
        term = a[n - 1][j] * minor
        cnt.mul += 1
        terms.append((cnt.mul, cnt.add))
        total_val = term if total_val is None else total_val + term
    sigma_add = n - 1
    tot_mul = sum(t[0] for t in terms)
    tot_add = sum(t[1] for t in terms) + sigma_add
    stored = sum(1 for (r, c) in store if r >= 1)
    return total_val, {"terms": terms, "sigma_add": sigma_add,
                       "total": (tot_mul, tot_add), "stored": stored}


def reference_multiplicity(n: int) -> Dict[int, Counter]:
    """How often each distinct minor is referenced in the un-stored expansion tree.

    Layer L (L = 1..n-1) holds the minors of order n-L that appear after L
    developments along the last remaining row (Section 4.2 and 4.3 call these
    "repeating terms").  Returns {L: Counter({multiplicity: number of distinct
    minors with that multiplicity})}, found by walking the full tree.
    """
    refs: Dict[int, Counter] = {}

    def walk(r: int, cols: FrozenSet[int], layer: int):
        if layer >= 1:
            refs.setdefault(layer, Counter())[cols] += 1
        if r == 0:
            return
        for j in sorted(cols):
            walk(r - 1, cols - {j}, layer + 1)

    walk(n - 1, frozenset(range(n)), 0)
    out: Dict[int, Counter] = {}
    for layer, c in refs.items():
        out[layer] = Counter(c.values())
    return out

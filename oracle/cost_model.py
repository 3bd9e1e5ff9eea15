"""Operation counts and the machine-time model (Su & Zheng, Sections 3.2, 3.3, 5.1, 5.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Naive (Section 3.2): n!(n-1) multiplications and n!-1 additions.
* Ryser (Section 3.3): (2^n - 1)(n - 1) multiplications and
  (2^n - n)(n + 1) - 2 additions; references [1][2] of the paper count the
  additions as (2^n - 2)(n + 1) instead (Section 3.3, the bracketed numbers of
  Tables 4 and 5).
* Store-zechin (Section 4): the counts come from the instrumented development
  in ``store_zechin.py`` (the paper gives no formula, Section 5.1).
* Time (Section 5.2): multiplications / multiply rate + additions / add rate,
  with ENIAC at 5000 additions/s and 357 multiplications/s and TRADIC at
  62500 additions/s and 3333 multiplications/s.  Reported in milliseconds.
"""
from __future__ import annotations

import math

from .store_zechin import store_zechin

MACHINES = {
    "ENIAC": {"add_per_s": 5000.0, "mul_per_s": 357.0},
    "TRADIC": {"add_per_s": 62500.0, "mul_per_s": 3333.0},
}


def naive_counts(n: int):
    return math.factorial(n) * (n - 1), math.factorial(n) - 1


def ryser_counts(n: int):
    return (2 ** n - 1) * (n - 1), (2 ** n - n) * (n + 1) - 2


def ryser_counts_refs12(n: int):
    return (2 ** n - 1) * (n - 1), (2 ** n - 2) * (n + 1)


def ryser_counts_instrumented(n: int):
    """Count the Ryser steps the way Section 3.3 describes them.

    Subsets are taken in ascending size; the row sums of a subset of size
    x+1 reuse those of a subset of size x (one addition per row), a
    size-1 subset's row sums are single entries (no addition), each product of
    n row sums takes n-1 multiplications, and the 2^n - 1 signed products are
    summed (2^n - 2 additions).
    """
    mul = add = 0
    for size in range(1, n + 1):
        count = math.comb(n, size)
        mul += count * (n - 1)
        if size >= 2:
            add += count * n
    add += (2 ** n - 1) - 1
    return mul, add


def store_zechin_counts(n: int):
    """Store-zechin (mul, add) from the instrumented development on a generic matrix."""
    a = [[1] * n for _ in range(n)]
    _, table = store_zechin(a)
    return table["total"]


def time_ms(mul: int, add: int, machine: str) -> float:
    r = MACHINES[machine]
    return 1000.0 * (mul / r["mul_per_s"] + add / r["add_per_s"])

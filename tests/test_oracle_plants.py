"""The oracle's pins catch plausible mistakes.

Each case builds a deliberately wrong variant of the C oracle (a dropped
low word, a wrong sign, a dropped term, a wrong index) on the CPU and checks
that at least one pin of tests/test_oracle.py fails against it."""
import ctypes
import math

import numpy as np
import pytest

import oracle


def _pins_hold():
    """A compact selection of the pins; returns False at the first violation."""
    try:
        if oracle.per_ryser(np.ones((5, 5), dtype=np.int64)) != math.factorial(5):
            return False
        if oracle.per_ryser(np.ones((6, 6), dtype=np.int64)) != math.factorial(6):
            return False
        if oracle.per_brute(np.array([[7, 0, 1, 2], [5, 3, 4, 5], [3, 5, 6, 7], [1, 7, 8, 9]])) != 9722:
            return False
        g = np.random.default_rng(5)
        n = 6
        x = g.standard_normal(n) + 1j * g.standard_normal(n)
        y = g.standard_normal(n) + 1j * g.standard_normal(n)
        want = math.factorial(n) * np.prod(x) * np.prod(y)
        got = oracle.dd_to_complex(oracle.per_ryser(np.outer(x, y)))
        if abs(got - want) > 1e-13 * abs(want):
            return False
        a = (1.0, 2.0 ** -60)
        b = (3.0, 2.0 ** -58)
        s = oracle.dd_add(a, b)
        from fractions import Fraction as F
        if abs(F(s[0]) + F(s[1]) - (F(1) + F(2.0 ** -60) + F(3) + F(2.0 ** -58))) > F(2) ** -100 * 4:
            return False
        return True
    except ValueError:
        return False


def test_correct_build_passes():
    assert _pins_hold()


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5])
def test_planted_mistake_is_caught(plant, tmp_path):
    path = oracle.build(out_path=str(tmp_path / f"liboracle_plant{plant}.so"),
                        defines=(f"ORACLE_PLANT={plant}",))
    bad = oracle._configure(ctypes.CDLL(path))
    old = oracle._swap_library(bad)
    try:
        assert not _pins_hold()
    finally:
        oracle._swap_library(old)

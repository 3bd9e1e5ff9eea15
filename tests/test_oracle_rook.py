"""Pins of oracle.rook (per(J - B) by rook numbers) against independent facts:
closed forms (n!, derangement numbers, a zero row, the full board's rook
numbers) and the permanent's definition (brute force over S_n, Eq. (1)) and
exact 256-bit Ryser (Eq. (4)) on random boards."""
import math

import numpy as np
import pytest

import oracle
from oracle.rook import complement_matrix, per_complement, rook_numbers


def derangements(n: int) -> int:
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[-1] + d[-2]))
    return d[n]


def random_board(n: int, size: int, seed: int):
    g = np.random.default_rng(seed)
    cells = set()
    while len(cells) < size:
        cells.add((int(g.integers(n)), int(g.integers(n))))
    return sorted(cells)


@pytest.mark.parametrize("n", [0, 1, 5, 12, 40])
def test_empty_board_is_factorial(n):
    assert per_complement(n, []) == math.factorial(n)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 12, 14])
def test_diagonal_board_is_derangements(n):
    assert per_complement(n, [(i, i) for i in range(n)]) == derangements(n)


def test_full_row_or_column_gives_zero():
    n = 9
    assert per_complement(n, [(4, j) for j in range(n)]) == 0
    assert per_complement(n, [(i, 2) for i in range(n)]) == 0


def test_full_board_rook_numbers():
    # k non-attacking rooks on the whole n x n board: C(n, k)^2 k!
    n = 4
    cells = [(i, j) for i in range(n) for j in range(n)]
    assert rook_numbers(cells) == [math.comb(n, k) ** 2 * math.factorial(k) for k in range(n + 1)] + [0] * (n * n - n)
    assert per_complement(n, cells) == 0


@pytest.mark.parametrize("n,size,seed", [(3, 2, 1), (5, 4, 2), (6, 9, 3), (7, 11, 4), (8, 14, 5), (8, 5, 6)])
def test_random_boards_against_brute_force(n, size, seed):
    cells = random_board(n, size, seed)
    assert per_complement(n, cells) == oracle.per_brute(complement_matrix(n, cells))


@pytest.mark.parametrize("n,size,seed", [(14, 12, 7), (17, 16, 8)])
def test_random_boards_against_exact_ryser(n, size, seed):
    cells = random_board(n, size, seed)
    assert per_complement(n, cells) == oracle.per_ryser(complement_matrix(n, cells))


def test_large_values_exceed_128_bits():
    # the regime the 192-bit GPU path is checked in: dense 0/1 matrices of order 35..40
    for n, seed in ((35, 11), (38, 12), (40, 13)):
        v = per_complement(n, random_board(n, 12, seed))
        assert 2 ** 128 < v < math.factorial(n) < 2 ** 160


@pytest.mark.parametrize("mistake", ["sign", "factorial", "attacking"])
def test_planted_mistakes_are_caught(mistake):
    """Plausible mistakes in the rook formula fail the pins above (derangements, brute force)."""
    from oracle import rook

    def wrong_rook_numbers(cells):
        # counts every subset of cells, attacking or not
        cs = sorted(set(cells))
        return [math.comb(len(cs), k) for k in range(len(cs) + 1)]

    def wrong(n, cells):
        r = wrong_rook_numbers(cells) if mistake == "attacking" else rook.rook_numbers(cells)
        total = 0
        for k, rk in enumerate(r):
            if k > n:
                continue
            sign = 1 if mistake == "sign" else (-1) ** k
            fact = math.factorial(n - k - 1) if (mistake == "factorial" and n - k >= 1) else math.factorial(n - k)
            total += sign * rk * fact
        return total

    caught = False
    for n in (3, 5, 7):
        if wrong(n, [(i, i) for i in range(n)]) != derangements(n):
            caught = True
    cells = random_board(6, 9, 3)
    if wrong(6, cells) != oracle.per_brute(complement_matrix(6, cells)):
        caught = True
    assert caught, mistake

"""Pins for the CPU oracle: values the paper prints, closed forms, invariants and
brute force on tiny inputs.  None of these compares the oracle with itself."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import cost_model as cm
from oracle.store_zechin import reference_multiplicity, store_zechin
from paper_1802_02779_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")
with open(GOLDEN) as f:
    PAPER = json.load(f)


def per3_textbook(m):
    """3x3 permanent written out: a(ei+fh) + b(di+fg) + c(dh+eg)."""
    (a, b, c), (d, e, f), (g, h, i) = m
    return a * (e * i + f * h) + b * (d * i + f * g) + c * (d * h + e * g)


def derangements(n):
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[k - 1] + d[k - 2]))
    return d[n]


def cplx(r):
    return oracle.dd_to_complex(r)


# --------------------------------------------------------------------------
# Section 3.1: the 4x4 worked development
# --------------------------------------------------------------------------

def test_paper_4x4_development():
    ex = PAPER["example_4x4"]
    A = np.array(ex["matrix"], dtype=np.int64)
    minors = [per3_textbook(m) for m in ex["minors"]]
    expected = sum(c * p for c, p in zip(ex["column0_coefficients"], minors))
    # the minors printed in the paper are A with row i and column 0 removed
    for i, m in enumerate(ex["minors"]):
        sub = np.delete(np.delete(A, i, axis=0), 0, axis=1)
        assert sub.tolist() == m
        assert oracle.per_brute(np.array(m)) == minors[i]
    assert minors == [1116, 258, 166, 122]
    assert expected == 9722
    assert oracle.per_brute(A) == expected
    assert oracle.per_ryser(A) == expected
    assert store_zechin(A.tolist())[0] == expected


# --------------------------------------------------------------------------
# closed forms and special matrices
# --------------------------------------------------------------------------

def test_2x2_and_3x3_closed_forms():
    g = np.random.default_rng(7)
    for _ in range(20):
        a = g.integers(-9, 10, size=(2, 2))
        assert oracle.per_brute(a) == a[0, 0] * a[1, 1] + a[0, 1] * a[1, 0]
        assert oracle.per_ryser(a) == a[0, 0] * a[1, 1] + a[0, 1] * a[1, 0]
        b = g.integers(-9, 10, size=(3, 3))
        assert oracle.per_brute(b) == per3_textbook(b.tolist())
        assert oracle.per_ryser(b) == per3_textbook(b.tolist())
    z = g.standard_normal((2, 2)) + 1j * g.standard_normal((2, 2))
    want = z[0, 0] * z[1, 1] + z[0, 1] * z[1, 0]
    assert abs(cplx(oracle.per_brute(z)) - want) < 1e-15
    assert abs(cplx(oracle.per_ryser(z)) - want) < 1e-15


def test_empty_and_1x1():
    assert oracle.per_brute(np.zeros((0, 0), dtype=np.int64)) == 1
    assert oracle.per_ryser(np.zeros((0, 0), dtype=np.int64)) == 1
    assert oracle.per_brute(np.array([[5]])) == 5
    assert oracle.per_ryser(np.array([[5]])) == 5
    assert cplx(oracle.per_ryser(np.array([[2 - 3j]]))) == 2 - 3j


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_identity_ones_derangements_brute(n):
    assert oracle.per_brute(np.eye(n, dtype=np.int64)) == 1
    assert oracle.per_brute(np.ones((n, n), dtype=np.int64)) == math.factorial(n)
    assert oracle.per_brute(np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64)) == derangements(n)


@pytest.mark.parametrize("n", [1, 3, 8, 13, 21])
def test_identity_ones_derangements_ryser(n):
    J = np.ones((n, n), dtype=np.int64)
    assert oracle.per_ryser(np.eye(n, dtype=np.int64)) == 1
    assert oracle.per_ryser(J) == math.factorial(n)
    assert oracle.per_ryser(J - np.eye(n, dtype=np.int64)) == derangements(n)


def test_d21_needs_more_than_64_bits():
    n = 21
    v = oracle.per_ryser(np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64))
    assert v == 18795307255050944540 and v >= 2 ** 64


def test_ones_matrix_beyond_128_bits():
    # 34! > 2^127: exercises the upper limbs of the 256-bit accumulator
    n = 22
    assert oracle.per_ryser(np.full((n, n), 3, dtype=np.int64)) == math.factorial(n) * 3 ** n


@pytest.mark.parametrize("n", [3, 6, 8])
def test_rank_one_complex_brute(n):
    g = np.random.default_rng(n)
    x = g.standard_normal(n) + 1j * g.standard_normal(n)
    y = g.standard_normal(n) + 1j * g.standard_normal(n)
    want = math.factorial(n) * np.prod(x) * np.prod(y)
    got = cplx(oracle.per_brute(np.outer(x, y)))
    assert abs(got - want) <= 1e-13 * abs(want)


@pytest.mark.parametrize("n", [4, 12, 18])
def test_rank_one_complex_ryser(n):
    g = np.random.default_rng(100 + n)
    x = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
    y = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
    want = math.factorial(n) * np.prod(x) * np.prod(y)
    scale = math.factorial(n) * np.prod(np.abs(x)) * np.prod(np.abs(y))   # per(|A|)
    got = cplx(oracle.per_ryser(np.outer(x, y)))
    assert abs(got - want) <= 1e-13 * scale


def test_triangular_and_block_diagonal():
    g = np.random.default_rng(3)
    for n in (4, 7, 11):
        t = np.triu(g.integers(1, 6, size=(n, n)))
        assert oracle.per_ryser(t) == int(np.prod(np.diag(t)))
    a = g.integers(0, 4, size=(3, 3))
    b = g.integers(0, 4, size=(4, 4))
    blk = np.zeros((7, 7), dtype=np.int64)
    blk[:3, :3] = a
    blk[3:, 3:] = b
    assert oracle.per_ryser(blk) == oracle.per_brute(a) * oracle.per_brute(b)
    za = g.standard_normal((3, 3)) + 1j * g.standard_normal((3, 3))
    zb = g.standard_normal((5, 5)) + 1j * g.standard_normal((5, 5))
    zblk = np.zeros((8, 8), dtype=np.complex128)
    zblk[:3, :3] = za
    zblk[3:, 3:] = zb
    want = cplx(oracle.per_brute(za)) * cplx(oracle.per_brute(zb))
    assert abs(cplx(oracle.per_ryser(zblk)) - want) <= 1e-13 * abs(want)


def test_zero_row_gives_zero():
    g = np.random.default_rng(4)
    a = g.integers(1, 5, size=(9, 9))
    a[4] = 0
    assert oracle.per_ryser(a) == 0
    assert oracle.per_brute(a) == 0


# --------------------------------------------------------------------------
# properties (1)-(3) of Section 3.1 on random inputs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [5, 8])
def test_properties_integer(n):
    g = np.random.default_rng(n)
    a = g.integers(0, 7, size=(n, n))
    p = oracle.per_brute(a)
    assert oracle.per_brute(a[g.permutation(n)]) == p           # (1) rows
    assert oracle.per_brute(a[:, g.permutation(n)]) == p        # (1) columns
    assert oracle.per_brute(a.T) == p                           # (2)
    b = a.copy()
    b[2] *= 5
    assert oracle.per_brute(b) == 5 * p                         # (3) row
    c = a.copy()
    c[:, 1] *= 3
    assert oracle.per_ryser(c) == 3 * p                         # (3) column


def test_properties_complex():
    n = 10
    g = np.random.default_rng(11)
    a = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / 3
    scale = oracle.per_abs(a)
    p = cplx(oracle.per_ryser(a))
    assert abs(cplx(oracle.per_ryser(a[g.permutation(n)][:, g.permutation(n)])) - p) <= 1e-14 * scale
    assert abs(cplx(oracle.per_ryser(a.T)) - p) <= 1e-14 * scale
    s = 0.5 - 2j
    b = a.copy()
    b[3] *= s
    assert abs(cplx(oracle.per_ryser(b)) - s * p) <= 1e-14 * abs(s) * scale


# --------------------------------------------------------------------------
# the oracle's algorithms agree on tiny inputs; the dd primitives are exact
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 4, 6, 8])
def test_brute_ryser_storezechin_agree_int(n):
    g = np.random.default_rng(50 + n)
    for _ in range(3):
        a = g.integers(0, 10, size=(n, n))
        b = oracle.per_brute(a)
        assert oracle.per_ryser(a) == b
        assert store_zechin(a.tolist())[0] == b


@pytest.mark.parametrize("n", [3, 5, 7])
def test_brute_ryser_storezechin_agree_complex(n):
    g = np.random.default_rng(60 + n)
    a = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    scale = abs(cplx(oracle.per_brute(np.abs(a).astype(complex))))
    b = cplx(oracle.per_brute(a))
    assert abs(cplx(oracle.per_ryser(a)) - b) <= 1e-15 * scale
    # exact rational Store-zechin on the same (binary) entries
    fa = [[(Fraction(float(z.real)), Fraction(float(z.imag))) for z in row] for row in a]

    class Q:
        def __init__(self, re, im):
            self.re, self.im = re, im

        def __mul__(self, o):
            return Q(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

        def __add__(self, o):
            return Q(self.re + o.re, self.im + o.im)

    qa = [[Q(*e) for e in row] for row in fa]
    ex = store_zechin(qa)[0]
    exact = complex(float(ex.re), float(ex.im))
    r = oracle.per_brute(a)
    # the dd result is within a few units of 2^-100 of the exact rational value
    err_re = abs(Fraction(r[0]) + Fraction(r[1]) - ex.re)
    err_im = abs(Fraction(r[2]) + Fraction(r[3]) - ex.im)
    assert float(err_re) <= 1e-28 * scale and float(err_im) <= 1e-28 * scale
    assert abs(b - exact) <= 1e-15 * scale


def test_dd_primitives_against_rationals():
    g = np.random.default_rng(12)
    for _ in range(300):
        a = (float(g.standard_normal()), 0.0)
        a = (a[0], a[0] * 2.0 ** -60 * float(g.random()))
        b = (float(g.standard_normal()) * 2.0 ** int(g.integers(-20, 20)), 0.0)
        b = (b[0], b[0] * 2.0 ** -58 * float(g.random()))
        A = Fraction(a[0]) + Fraction(a[1])
        B = Fraction(b[0]) + Fraction(b[1])
        s = oracle.dd_add(a, b)
        m = oracle.dd_mul(a, b)
        assert abs(Fraction(s[0]) + Fraction(s[1]) - (A + B)) <= Fraction(2) ** -100 * (abs(A) + abs(B))
        assert abs(Fraction(m[0]) + Fraction(m[1]) - A * B) <= Fraction(2) ** -100 * abs(A * B)


# --------------------------------------------------------------------------
# Section 4 and 5: operation counts and the machine-time model
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", ["3", "4", "5"])
def test_store_zechin_tables_1_to_3(n):
    want = PAPER["store_zechin_tables"][n]
    _, t = store_zechin([[1] * int(n) for _ in range(int(n))])
    assert [list(x) for x in t["terms"]] == want["terms"]
    assert t["sigma_add"] == want["sigma"][1]
    assert list(t["total"]) == want["total"]


def test_repeating_terms():
    for n, layers in PAPER["repeating_terms"].items():
        if n.startswith("_"):
            continue
        mult = reference_multiplicity(int(n))
        for layer, spec in layers.items():
            assert mult[int(layer)] == {spec["fold"]: spec["count"]}
    # n = 3: every minor referenced once ("no repeating term", Section 4.1)
    m3 = reference_multiplicity(3)
    assert set(m3[1]) == {1}


@pytest.mark.parametrize("n", range(2, 9))
def test_store_zechin_closed_forms(n):
    mul, add = cm.store_zechin_counts(n)
    assert mul == n * (2 ** (n - 1) - 1)
    assert add == (n - 2) * 2 ** (n - 1) + 1
    # every k-subset of columns is stored exactly once (k = 2..n-1)
    _, t = store_zechin([[1] * n for _ in range(n)])
    assert t["stored"] == sum(math.comb(n, k) for k in range(2, n))


def test_table4():
    t4 = PAPER["table4"]
    for n in ("3", "4", "5"):
        k = int(n)
        assert list(cm.naive_counts(k)) == t4["Naive"][n]
        assert list(cm.ryser_counts(k)) == t4["Ryser"][n]
        assert list(cm.ryser_counts_instrumented(k)) == t4["Ryser"][n]
        assert cm.ryser_counts_refs12(k)[1] == t4["Ryser_refs12_add"][n]
        assert list(cm.store_zechin_counts(k)) == t4["Store-zechin"][n]


def test_table5():
    t5 = PAPER["table5_ms"]
    rates = PAPER["machine_rates"]
    for machine in ("ENIAC", "TRADIC"):
        assert cm.MACHINES[machine]["add_per_s"] == rates[machine]["add_per_s"]
        assert cm.MACHINES[machine]["mul_per_s"] == rates[machine]["mul_per_s"]
        for i, n in enumerate((3, 4, 5)):
            for name, counts in (("Naive", cm.naive_counts(n)), ("Ryser", cm.ryser_counts(n)),
                                 ("Ryser_refs12", cm.ryser_counts_refs12(n)),
                                 ("Store-zechin", cm.store_zechin_counts(n))):
                got = cm.time_ms(counts[0], counts[1], machine)
                # printed to 0.1 ms; one entry (bracketed Ryser, ENIAC, n=4: 140.05)
                # is printed as 140.0, i.e. truncated rather than rounded
                assert abs(got - t5[name][machine][i]) < 0.051, (name, machine, n, got)
                if (name, machine, n) != ("Ryser_refs12", "ENIAC", 4):
                    assert round(got, 1) == pytest.approx(t5[name][machine][i], abs=1e-9)


# --------------------------------------------------------------------------
# Section 2: amplitudes of a unitary form a probability distribution
# --------------------------------------------------------------------------

def test_boson_sampling_sum_rule():
    m, n = 9, 5
    u = wl.haar_unitary(m, 18021)
    total = 0.0
    for t in itertools.combinations_with_replacement(range(m), n):
        sub = u[:n][:, list(t)]
        p = cplx(oracle.per_brute(sub))
        mult = 1
        for c in set(t):
            mult *= math.factorial(t.count(c))
        total += abs(p) ** 2 / mult
    assert abs(total - 1.0) < 1e-12


def test_haar_is_unitary():
    u = wl.haar_unitary(40, 5)
    assert np.allclose(u.conj().T @ u, np.eye(40), atol=1e-12)

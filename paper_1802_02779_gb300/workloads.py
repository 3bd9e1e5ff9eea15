"""Seeded synthetic inputs for permanent computations.

This module only makes inputs; it contains none of the permanent arithmetic,
and both the GPU path and the CPU oracle draw their inputs from it.

Boson-sampling inputs follow Section 2 of Su & Zheng (arXiv:1802.02779): an
amplitude is proportional to the permanent of the n x n submatrix of an m x m
unitary U that keeps the n input rows and the n output columns.  The paper
names no distribution for U; a Haar-random unitary is used (complex Gaussian
with independent N(0, 1/2) real and imaginary parts, QR, then every column
multiplied by the phase of the matching diagonal entry of R, Mezzadri,
Notices AMS 54 (2007)).  Integer inputs are Bernoulli 0/1 matrices, the
#P-complete case Section 2 mentions.

Every generator takes an explicit seed and uses numpy's PCG64.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import List

import numpy as np

SEED_BASE = 18020


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar_unitary(m: int, seed: int) -> np.ndarray:
    """Haar-random m x m unitary (complex128)."""
    g = rng(seed)
    z = (g.standard_normal((m, m)) + 1j * g.standard_normal((m, m))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return (q * ph[None, :]).astype(np.complex128)


def submatrix(u: np.ndarray, rows, cols) -> np.ndarray:
    return np.ascontiguousarray(u[np.ix_(list(rows), list(cols))])


def bernoulli01(count: int, n: int, p, seed: int) -> np.ndarray:
    """count x n x n int64 0/1 matrices; p is one density or one per matrix."""
    g = rng(seed)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), (count,))
    u = g.random((count, n, n))
    return (u < p[:, None, None]).astype(np.int64)


def gaussian_complex(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """n x n i.i.d. complex Gaussian, E|z|^2 = 1, times `scale`."""
    g = rng(seed)
    z = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2.0)
    return (z * scale).astype(np.complex128)


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------

def five_boson(seed_u: int = SEED_BASE + 1, seed_b: int = SEED_BASE + 2):
    """5-boson sampling: rows 0..4 of a 9x9 Haar unitary, all C(9,5)=126
    collision-free output patterns in lexicographic order, plus 100 Bernoulli(0.5)
    5x5 0/1 matrices.  Returns (complex (126,5,5), int64 (100,5,5))."""
    u = haar_unitary(9, seed_u)
    rows = range(5)
    cmats = np.stack([submatrix(u, rows, cols) for cols in itertools.combinations(range(9), 5)])
    imats = bernoulli01(100, 5, 0.5, seed_b)
    return cmats, imats


def batched_n20(count: int = 4096, seed_u: int = SEED_BASE + 3, seed_b: int = SEED_BASE + 4,
                n: int = 20, m: int = 400):
    """count n x n submatrices of an m x m Haar unitary (rows 0..n-1, a uniformly
    random sorted n-subset of the m columns each) and count Bernoulli(0.5) n x n
    0/1 matrices.  Returns (complex (count,n,n), int64 (count,n,n))."""
    u = haar_unitary(m, seed_u)
    g = rng(seed_u + 1000)
    cmats = np.empty((count, n, n), dtype=np.complex128)
    for i in range(count):
        cols = np.sort(g.choice(m, size=n, replace=False))
        cmats[i] = u[:n][:, cols]
    imats = bernoulli01(count, n, 0.5, seed_b)
    return cmats, imats


def single_n32(seed: int = SEED_BASE + 5, n: int = 32) -> np.ndarray:
    """One n x n i.i.d. complex Gaussian matrix scaled by 1/sqrt(n*n) (E|z|^2 = 1 before scaling)."""
    return gaussian_complex(n, seed, scale=1.0 / np.sqrt(n * n))


@dataclass
class Request:
    n: int
    dtype: str          # "c128" or "u01"
    mat: np.ndarray
    arrival_s: float = 0.0


def uneven_requests(count: int = 20000, seed: int = SEED_BASE + 6, seed_u: int = SEED_BASE + 7,
                    n_lo: int = 8, n_hi: int = 28, frac_complex: float = 0.7,
                    m: int = 256) -> List[Request]:
    """count requests, n uniform in [n_lo, n_hi]; frac_complex are submatrices
    of an m x m Haar unitary (rows 0..n-1, random sorted n-subset of columns),
    the rest 0/1 with a per-matrix density uniform in [0.3, 0.7]."""
    u = haar_unitary(m, seed_u)
    g = rng(seed)
    out: List[Request] = []
    for _ in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        if g.random() < frac_complex:
            cols = np.sort(g.choice(m, size=n, replace=False))
            out.append(Request(n, "c128", np.ascontiguousarray(u[:n][:, cols])))
        else:
            p = g.uniform(0.3, 0.7)
            mat = (g.random((n, n)) < p).astype(np.int64)
            out.append(Request(n, "u01", mat))
    return out


def poisson_arrivals(count: int, rate_per_s: float, seed: int = SEED_BASE + 8,
                     n_lo: int = 10, n_hi: int = 36, frac_complex: float = 0.7,
                     m: int = 256, seed_u: int = SEED_BASE + 7) -> List[Request]:
    """Serving workload: Poisson arrivals at `rate_per_s`, n uniform in
    [n_lo, n_hi], mix as in :func:`uneven_requests`."""
    reqs = uneven_requests(count, seed=seed, seed_u=seed_u, n_lo=n_lo, n_hi=n_hi,
                           frac_complex=frac_complex, m=m)
    g = rng(seed + 500)
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    for r, ti in zip(reqs, t):
        r.arrival_s = float(ti)
    return reqs


def concat(mats) -> np.ndarray:
    """Concatenate matrices of mixed order into one flat array (row-major each)."""
    return np.concatenate([np.ascontiguousarray(m).reshape(-1) for m in mats]) if len(mats) else np.zeros(0)

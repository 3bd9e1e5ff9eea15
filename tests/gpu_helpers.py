"""Shared helpers for the GPU parity tests (host side only)."""
import numpy as np

import oracle


def oracle_c(m) -> complex:
    return oracle.dd_to_complex(oracle.per_brute(m) if m.shape[0] <= 8 else oracle.per_ryser(m))


def oracle_i(m) -> int:
    return oracle.per_brute(m) if m.shape[0] <= 8 else oracle.per_ryser(m)


def tol_c(m) -> float:
    """The tolerance for complex results: 1e-12 * per(|A|)."""
    return 1e-12 * oracle.per_abs(m)


def rand_complex(n, seed, scale=None):
    g = np.random.default_rng(seed)
    z = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2.0)
    return z * (scale if scale is not None else 1.0 / np.sqrt(max(n, 1)))


def rand01(n, seed, p=0.5):
    g = np.random.default_rng(seed)
    return (g.random((n, n)) < p).astype(np.int64)

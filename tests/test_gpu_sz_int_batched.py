"""The batched integer Store-zechin kernel (one CTA per matrix) against the oracle.

A call takes the batched kernel only when it holds at least as many
Store-zechin matrices as the GPU has SMs, so every call here repeats a set of
matrices to fill it.  Covered: 0/1 matrices of order <= 20 (the register-row
kernel, 64-bit chains; orders 1 and 2 and chain widths below 3 on the mask-list
chains), 0/1 matrices of order 21..23 (64- and 128-bit chains chosen per
matrix), small nonnegative integers (multiply-add, 64 and 128 bits), chain
widths 3..13 (fewer than five low columns: partial warp tasks; 13: two passes
of the outer phase) and CTAs of 256 and 512 threads.  Every value is exact."""
import math

import numpy as np
import pytest

from tests.gpu_helpers import oracle_i, rand01

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp():
    assert torch.cuda.is_available()
    from paper_1802_02779_gb300 import build
    build.build()
    from paper_1802_02779_gb300 import libperm
    libperm.load()
    return libperm


def _fill(lp, mats):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    reps = (sms + len(mats) - 1) // len(mats) + 1
    return [m for _ in range(reps) for m in mats]


def _run(lp, mats, dtype, **plan_kw):
    full = _fill(lp, mats)
    with lp.Plan(max(m.shape[0] for m in full), dtype, method=lp.METHOD_SZ, max_batch=len(full),
                 **plan_kw) as p:
        got, st = lp.permanents(full, dtype, plan=p, return_status=True)
    assert (np.asarray(st) == lp.PERM_OK).all()
    k = len(mats)
    for r in range(1, len(full) // k):          # every repeat of a matrix gives the same value
        assert got[r * k:(r + 1) * k] == got[:k]
    return got[:k]


@pytest.mark.parametrize("low_cols", [0, 3, 5, 7, 11, 13])
def test_01_orders_up_to_20(lp, low_cols):
    mats = [rand01(n, 12000 + n, p=0.55) for n in (1, 2, 4, 6, 9, 12, 15, 17, 19, 20)]
    got = _run(lp, mats, "u01", low_cols=low_cols)
    assert got == [oracle_i(m) for m in mats]


def test_01_closed_forms_and_128_bits(lp):
    """J_n = n! and J - I = D_n for n = 20..23 (21! > 2^64: 128-bit chains)."""
    mats, want = [], []
    for n in range(20, 24):
        J = np.ones((n, n), dtype=np.int64)
        mats += [J, J - np.eye(n, dtype=np.int64)]
        d = [1, 0]
        for k in range(2, n + 1):
            d.append((k - 1) * (d[-1] + d[-2]))
        want += [math.factorial(n), d[n]]
    mats.append(rand01(22, 12100, p=0.5))
    want.append(oracle_i(mats[-1]))
    assert _run(lp, mats, "u01") == want


@pytest.mark.parametrize("low_cols", [0, 3, 12, 13])
def test_01_register_rows_closed_forms(lp, low_cols):
    """0/1 batches of order <= 20 (the register-row kernel) on matrices with closed forms:
    J_n = n!, J - I = D_n, a zero row or column = 0, a permutation matrix = 1, an upper
    triangular matrix of ones = 1, and a block-diagonal matrix = the product of its blocks."""
    mats, want = [], []
    d = [1, 0]
    for k in range(2, 21):
        d.append((k - 1) * (d[-1] + d[-2]))
    for n in (3, 7, 13, 19, 20):
        J = np.ones((n, n), dtype=np.int64)
        mats += [J, J - np.eye(n, dtype=np.int64)]
        want += [math.factorial(n), d[n]]
    z = rand01(18, 12400, p=0.6)
    z[11, :] = 0
    mats.append(z); want.append(0)
    z = rand01(20, 12401, p=0.6)
    z[:, 19] = 0
    mats.append(z); want.append(0)
    perm = np.random.default_rng(12402).permutation(20)
    mats.append(np.eye(20, dtype=np.int64)[perm]); want.append(1)
    mats.append(np.triu(np.ones((20, 20), dtype=np.int64))); want.append(1)
    b1, b2 = rand01(9, 12403, p=0.5), rand01(11, 12404, p=0.5)
    blk = np.zeros((20, 20), dtype=np.int64)
    blk[:9, :9] = b1
    blk[9:, 9:] = b2
    mats.append(blk); want.append(oracle_i(b1) * oracle_i(b2))
    assert _run(lp, mats, "u01", low_cols=low_cols) == want


@pytest.mark.parametrize("low_cols", [0, 4, 12])
def test_small_integers_multiply_add(lp, low_cols):
    g = np.random.default_rng(12200)
    mats = [g.integers(0, 4, size=(n, n)).astype(np.int64) for n in (3, 8, 12, 16, 18)]
    big = np.full((17, 17), 9, dtype=np.int64)            # 9^17 * 17! > 2^64: 128 bits
    mats.append(big)
    got = _run(lp, mats, "i64", low_cols=low_cols)
    assert got[:-1] == [oracle_i(m) for m in mats[:-1]]
    assert got[-1] == 9 ** 17 * math.factorial(17)


@pytest.mark.parametrize("low_cols", [0, 13])
def test_512_thread_ctas(lp, monkeypatch, low_cols):
    """The other CTA size of the integer kernel (512 threads, which the autotuner
    may pick) gives the same values."""
    monkeypatch.setenv("LIBPERM_SZ_THREADS", "512")
    mats = [rand01(n, 12300 + n, p=0.5) for n in (10, 16, 20)]
    mats.append(np.full((12, 12), 3, dtype=np.int64))
    with lp.Plan(20, "u01", method=lp.METHOD_SZ) as p:
        assert p.describe()["cta_threads"] == 512
    got = _run(lp, mats[:3], "u01", low_cols=low_cols)
    assert got == [oracle_i(m) for m in mats[:3]]
    assert _run(lp, mats[3:], "i64", low_cols=low_cols) == [3 ** 12 * math.factorial(12)]

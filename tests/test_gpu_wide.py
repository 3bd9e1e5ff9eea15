"""GPU: exact integer permanents above 2^128 (PERM_FLAG_WIDE: 256-bit result
slots, Ryser modulo 2^192) and the integer routing of PERM_METHOD_AUTO.

Expected values come from closed forms (n!, c^n n!, rank one), from the
rook-number oracle (per(J - B), oracle.rook) and from the exact 256-bit Ryser
oracle; every comparison is exact."""
import math

import numpy as np
import pytest

import oracle
from oracle.rook import complement_matrix, per_complement
from tests.gpu_helpers import rand01, rand_complex

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1802_02779_gb300 import build
    build.build()
    from paper_1802_02779_gb300 import libperm
    libperm.load()
    return libperm


def wide(lp, mats, dtype, method=None):
    return lp.permanents(mats, dtype, method=lp.METHOD_AUTO if method is None else method,
                         flags=lp.FLAG_WIDE, return_status=True)


def random_board(n, size, seed):
    g = np.random.default_rng(seed)
    cells = set()
    while len(cells) < size:
        cells.add((int(g.integers(n)), int(g.integers(n))))
    return sorted(cells)


def test_ones_matrices_35_to_40(lp):
    ns = [35, 36, 40]
    res, st = wide(lp, [np.ones((n, n), np.int64) for n in ns], "u01")
    assert list(st) == [lp.PERM_OK] * len(ns)
    assert res == [math.factorial(n) for n in ns]


def test_without_wide_the_status_reports_overflow(lp):
    res, st = lp.permanents([np.ones((36, 36), np.int64)], "u01", return_status=True)
    assert list(st) == [lp.PERM_EOVERFLOW]
    assert res[0] == math.factorial(36) % 2 ** 128


@pytest.mark.parametrize("n,size,seed", [(35, 10, 1), (36, 14, 2), (37, 8, 3), (38, 12, 4)])
def test_dense_01_against_rook_numbers(lp, n, size, seed):
    cells = random_board(n, size, seed)
    want = per_complement(n, cells)
    assert want > 2 ** 128
    res, st = wide(lp, [complement_matrix(n, cells)], "u01")
    assert st[0] == lp.PERM_OK and res[0] == want


def test_scaled_ones_i64(lp):
    # 2 J_30: per = 2^30 30! ~ 2^138; the row-sum bound 60^30 ~ 2^177 selects 192 bits
    n = 30
    res, st = wide(lp, [np.full((n, n), 2, np.int64)], "i64")
    assert st[0] == lp.PERM_OK and res[0] == 2 ** 30 * math.factorial(n)


def test_rank_one_i64(lp):
    # per(x y^T) = n! prod x prod y: here ~2^140 and ~2^147, bounds ~2^172 and ~2^180
    g = np.random.default_rng(5)
    mats, want = [], []
    for n in (24, 25):
        x = g.integers(2, 4, n)
        y = g.integers(2, 4, n)
        mats.append(np.outer(x, y).astype(np.int64))
        want.append(math.factorial(n) * math.prod(int(v) for v in x) * math.prod(int(v) for v in y))
    res, st = wide(lp, mats, "i64")
    assert list(st) == [lp.PERM_OK] * 2
    assert res == want
    assert min(want) > 2 ** 128


def test_small_ints_against_exact_ryser_oracle(lp):
    # entries 0..9: n = 20 has a bound above 2^128 (192-bit path, value below 2^128),
    # n = 24 has a value above 2^128
    g = np.random.default_rng(21)
    mats = [g.integers(0, 10, (20, 20)).astype(np.int64) for _ in range(2)]
    mats += [g.integers(0, 10, (24, 24)).astype(np.int64)]
    res, st = wide(lp, mats, "i64")
    assert list(st) == [lp.PERM_OK] * 3
    want = [oracle.per_ryser(m) for m in mats]
    assert res == want
    assert want[2] > 2 ** 128


def test_wide_and_narrow_results_agree(lp):
    mats = [rand01(n, 300 + n) for n in (5, 12, 20, 24, 28)] + [np.zeros((0, 0), np.int64)]
    a, sa = lp.permanents(mats, "u01", return_status=True)
    b, sb = wide(lp, mats, "u01")
    assert a == b and list(sa) == list(sb)


@pytest.mark.parametrize("method", ["auto", "sz"])
def test_wide_slots_layout(lp, method):
    """Four words per matrix, the high ones zero below 2^128; n = 0 gives (1, 0, 0, 0)."""
    m = lp.METHOD_SZ if method == "sz" else lp.METHOD_AUTO
    mats = [rand01(n, 400 + n) for n in (6, 14, 20, 23)] + [np.zeros((0, 0), np.int64)]
    sizes = [a.shape[0] for a in mats]
    flat = np.concatenate([a.reshape(-1) for a in mats])
    dev = torch.from_numpy(flat).cuda()
    out = torch.full((len(mats), 4), -1, dtype=torch.int64, device="cuda")
    st = torch.full((len(mats),), -1, dtype=torch.int32, device="cuda")
    with lp.Plan(23, "u01", method=m, flags=lp.FLAG_WIDE) as p:
        assert p.describe()["out_words"] == 4
        p.batch(dev, sizes, out, st)
        torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert (st.cpu().numpy() == lp.PERM_OK).all()
    assert (o[:, 2:] == 0).all()
    assert list(o[-1]) == [1, 0, 0, 0]
    assert [lp.words_to_int(r) for r in o[:-1]] == lp.permanents(mats[:-1], "u01")


def test_store_zechin_stays_128_bits(lp):
    # Store-zechin's tables are at most 128 bits wide: above that it reports overflow
    n = 24
    a = np.full((n, n), 3, np.int64)      # 3^24 24! ~ 2^117 fits, bound 72^24 ~ 2^148 does not
    res, st = wide(lp, [a], "i64", method=lp.METHOD_SZ)
    assert st[0] == lp.PERM_EOVERFLOW
    assert res[0] == (3 ** n * math.factorial(n)) % 2 ** 128
    res, st = wide(lp, [a], "i64")
    assert st[0] == lp.PERM_OK and res[0] == 3 ** n * math.factorial(n)


def test_wide_rejected_for_complex(lp):
    with pytest.raises(lp.LibpermError) as e:
        lp.Plan(5, "c128", flags=lp.FLAG_WIDE)
    assert e.value.status == lp.PERM_EINVAL


def test_auto_routes_integers_to_ryser(lp):
    with lp.Plan(24, "u01") as p:
        d = p.describe()
        assert d["sz_batch_nmax"] == 0 and d["sz_single_nmax"] == 0
    with lp.Plan(24, "c128") as p:
        assert p.describe()["sz_single_nmax"] == 24


def test_server_wide(lp):
    c5 = rand_complex(5, 77)
    with lp.Server(flags=lp.FLAG_WIDE) as srv:
        ts = [srv.submit(np.ones((36, 36), np.int64), "u01"),
              srv.submit(np.ones((5, 5), np.int64), "u01"),
              srv.submit(c5, "c128"),
              srv.submit(np.full((30, 30), 2, np.int64), "i64")]
        res = srv.wait_all(ts, timeout_s=600)
    assert res[0] == (math.factorial(36), lp.PERM_OK)
    assert res[1] == (120, lp.PERM_OK)
    assert res[2][0] == lp.permanents([c5], "c128")[0] and res[2][1] == lp.PERM_OK
    assert res[3] == (2 ** 30 * math.factorial(30), lp.PERM_OK)


# ---------------------------------------------------------------------------
# 0/1 Ryser by Glynn's formula modulo 2^(w + n - 1), shifted by n - 1
# ---------------------------------------------------------------------------
def test_glynn_ones_every_order(lp):
    ns = list(range(1, 35))
    res, st = lp.permanents([np.ones((n, n), np.int64) for n in ns], "u01", return_status=True)
    assert list(st) == [lp.PERM_OK] * len(ns)
    assert res == [math.factorial(n) for n in ns]


def test_glynn_against_store_zechin(lp):
    mats = [rand01(n, 500 + n, p=0.3 + 0.4 * (n % 3) / 2) for n in range(1, 25)]
    auto = lp.permanents(mats, "u01")
    sz = lp.permanents(mats, "u01", method=lp.METHOD_SZ)
    assert auto == sz


@pytest.mark.parametrize("n,size,seed", [(28, 9, 11), (31, 16, 12), (34, 10, 13)])
def test_glynn_128_against_rook_numbers(lp, n, size, seed):
    cells = random_board(n, size, seed)
    want = per_complement(n, cells)
    assert 2 ** 64 < want < 2 ** 128
    res, st = lp.permanents([complement_matrix(n, cells)], "u01", return_status=True)
    assert st[0] == lp.PERM_OK and res[0] == want


@pytest.mark.parametrize("n,hi,seed", [(7, 4, 1), (12, 4, 2), (16, 3, 3), (20, 2, 4),   # row sums <= 127
                                       (8, 1000, 5), (10, 1000, 6),                   # <= 32767
                                       (6, 100000, 7)])                               # Eq. 4 (larger)
def test_small_int_glynn_classes(lp, n, hi, seed):
    g = np.random.default_rng(seed)
    mats = [g.integers(0, hi + 1, (n, n)).astype(np.int64) for _ in range(3)]
    res, st = lp.permanents(mats, "i64", return_status=True)
    assert list(st) == [lp.PERM_OK] * 3
    assert res == [oracle.per_brute(m) if n <= 8 else oracle.per_ryser(m) for m in mats]
    assert res == lp.permanents(mats, "i64", method=lp.METHOD_SZ)

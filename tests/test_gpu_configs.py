"""The five workloads end to end through the C ABI, against the oracle.

* 5-boson (all 126 patterns + 100 0/1): tests/test_gpu_parity.py.
* batched n = 20: the full 4096 + 4096 batch in the launch configuration the
  bench times (autotuned plan); a seeded sample of outputs against the oracle,
  every status OK.
* single n = 32: Store-zechin and Ryser against the stored oracle value.
* uneven n = 8..28: the first 200 requests, every one against the oracle
  (n <= 22 computed here, n = 23..28 stored in tests/golden/); general complex
  n = 29..31 from the serving stream against stored oracle values.
* serving: the same matrix alone and through the server, including Ryser-lane
  orders (n = 34).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1802_02779_gb300 import workloads as wl
from tests.gpu_helpers import oracle_c, oracle_i, tol_c

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "single_n32.json")


@pytest.fixture(scope="module")
def lp():
    assert torch.cuda.is_available()
    from paper_1802_02779_gb300 import build
    build.build()
    from paper_1802_02779_gb300 import libperm
    libperm.load()
    return libperm


def test_batched_n20_full_batch_sampled(lp):
    cm, im = wl.batched_n20()
    count = cm.shape[0]
    sample = np.random.default_rng(20).choice(count, size=12, replace=False)
    for dt, mats in (("c128", cm), ("u01", im)):
        dev = torch.from_numpy(np.ascontiguousarray(mats).reshape(-1)).cuda()
        out = torch.empty(count, dtype=torch.complex128, device="cuda") if dt == "c128" else \
            torch.empty((count, 2), dtype=torch.int64, device="cuda")
        st = torch.empty(count, dtype=torch.int32, device="cuda")
        with lp.Plan(20, dt, max_batch=count, flags=lp.FLAG_AUTOTUNE) as p:
            p.batch(dev, [20] * count, out, st)
            torch.cuda.synchronize()
        assert int(st.abs().sum()) == 0
        o = out.cpu().numpy()
        for i in sample:
            if dt == "c128":
                assert abs(o[i] - oracle_c(mats[i])) <= tol_c(mats[i])
            else:
                assert lp.u128_to_int(o[i]) == oracle_i(mats[i])


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="tests/golden/single_n32.json not generated")
@pytest.mark.parametrize("method", ["sz", "ryser"])
def test_single_n32_against_stored_oracle(lp, method):
    g = json.load(open(GOLDEN))
    a = wl.single_n32()
    m = lp.METHOD_SZ if method == "sz" else lp.METHOD_RYSER
    got = lp.permanents([a], "c128", method=m)[0]
    want = complex(*g["per"])
    assert abs(got - want) <= 1e-12 * g["per_abs"], (got, want, g["per_abs"])


def _golden(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


@pytest.mark.parametrize("method", ["auto", "ryser"])
def test_uneven_sample(lp, method):
    """The first 200 requests of the uneven-size stream, batched by dtype as the
    stream delivers them: n <= 22 against the oracle computed here, every
    request of order 23..28 against the oracle's stored values
    (tests/golden/make_large_complex.py, tests/golden/make_large_u01.py)."""
    reqs = wl.uneven_requests(count=200)
    gc = {c["index"]: c for c in _golden("large_complex.json")["cases"] if c["stream"] == "uneven"}
    gi = {c["index"]: c for c in _golden("large_u01.json")["cases"]}
    m = lp.METHOD_AUTO if method == "auto" else lp.METHOD_RYSER
    for dt in ("c128", "u01"):
        idx = [i for i, r in enumerate(reqs) if r.dtype == dt]
        mats = [reqs[i].mat for i in idx]
        res, st = lp.permanents(mats, dt, method=m, return_status=True)
        assert (np.asarray(st) == lp.PERM_OK).all()
        for k, i in enumerate(idx):
            a = mats[k]
            if a.shape[0] <= 22:
                if method == "ryser" and k % 4:
                    continue                 # the Ryser pass samples a quarter of the small orders
                if dt == "c128":
                    assert abs(res[k] - oracle_c(a)) <= tol_c(a), (i, a.shape[0])
                else:
                    assert res[k] == oracle_i(a), (i, a.shape[0])
            elif dt == "c128":
                g = gc[i]                    # every large complex request has a stored value
                assert g["n"] == a.shape[0]
                want = complex(*g["per"])
                assert abs(res[k] - want) <= 1e-12 * g["per_abs"], (i, g["n"], res[k], want)
            else:
                g = gi[i]
                assert g["n"] == a.shape[0]
                assert res[k] == int(g["per"]), (i, g["n"])


@pytest.mark.parametrize("method", ["sz", "ryser"])
def test_serving_stream_orders_29_to_31(lp, method):
    """General complex matrices of order 29, 30 and 31 from the serving stream,
    one plan per order, against the oracle's stored double-double values."""
    gold = _golden("large_complex.json")
    kw = gold["streams"]["serving"]
    reqs = wl.uneven_requests(**kw)
    cases = [c for c in gold["cases"] if c["stream"] == "serving"]
    assert sorted(c["n"] for c in cases) == [29, 30, 31]
    m = lp.METHOD_SZ if method == "sz" else lp.METHOD_RYSER
    for c in cases:
        a = reqs[c["index"]].mat
        assert a.shape == (c["n"], c["n"]) and reqs[c["index"]].dtype == "c128"
        got = lp.permanents([a], "c128", method=m)[0]
        want = complex(*c["per"])
        assert abs(got - want) <= 1e-12 * c["per_abs"], (c["n"], got, want)


def test_serving_alone_vs_mix_large_orders(lp):
    g = np.random.default_rng(34)
    a34 = (g.standard_normal((34, 34)) + 1j * g.standard_normal((34, 34))) / (34 * np.sqrt(2))
    b26 = (g.random((26, 26)) < 0.5).astype(np.int64)
    small = [wl.gaussian_complex(12, 100 + k, scale=1 / 12) for k in range(20)]
    with lp.Server(mem_budget_bytes=8 << 30) as srv:
        t34 = srv.submit(a34, "c128")            # tables do not fit 8 GB: Ryser lane
        t26 = srv.submit(b26, "u01")             # integers: Ryser lane
        ts = [srv.submit(m, "c128") for m in small]
        res = srv.wait_all([t34, t26] + ts, timeout_s=600)
    assert all(st == lp.PERM_OK for _, st in res)
    assert res[0][0] == lp.permanents([a34], "c128", method=lp.METHOD_RYSER)[0]
    assert res[1][0] == lp.permanents([b26], "u01")[0]
    alone = lp.permanents(small, "c128")
    assert [r[0] for r in res[2:]] == list(alone)


@pytest.mark.parametrize("n,budget_gb", [(33, 60), (34, 100), (35, 200)])
def test_store_zechin_compact_tables(lp, n, budget_gb):
    """Orders 33..35 keep compact chain tables (Re, Im of each entry; w = Re + Im
    recomputed for outer terms): n = 35 needs 185 GB.  Pinned by the oracle through
    a block-diagonal matrix, per(B + C) = per(B) per(C), and by the rank-one closed
    form per(x y^T) = n! prod x prod y."""
    import math
    h = n // 2
    g = np.random.default_rng(3500 + n)
    b = (g.standard_normal((h, h)) + 1j * g.standard_normal((h, h))) / np.sqrt(2 * h)
    c = (g.standard_normal((n - h, n - h)) + 1j * g.standard_normal((n - h, n - h))) / np.sqrt(2 * (n - h))
    blk = np.zeros((n, n), dtype=np.complex128)
    blk[:h, :h] = b
    blk[h:, h:] = c
    x = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
    y = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
    r1 = np.outer(x, y)
    with lp.Plan(n, "c128", method=lp.METHOD_SZ, max_batch=2, mem_budget_bytes=budget_gb << 30) as p:
        d = p.describe()
        assert d["sz_single_nmax"] == n
        assert p.workspace_bytes() < (budget_gb << 30)
        got, st = lp.permanents([blk, r1], "c128", plan=p, return_status=True)
    assert list(st) == [lp.PERM_OK, lp.PERM_OK]
    want_blk = oracle_c(b) * oracle_c(c)
    scale_blk = oracle.per_abs(b) * oracle.per_abs(c)
    assert abs(got[0] - want_blk) <= 1e-12 * scale_blk, (got[0], want_blk)
    want_r1 = math.factorial(n) * np.prod(x) * np.prod(y)
    scale_r1 = math.factorial(n) * np.prod(np.abs(x)) * np.prod(np.abs(y))
    assert abs(got[1] - want_r1) <= 1e-12 * scale_r1, (got[1], want_r1)


def test_store_zechin_n34_in_hbm(lp):
    """n = 34 complex in compact chain tables (92 GB of HBM, a 150 GB budget).
    Pinned by the oracle through a block-diagonal matrix, per(B + C) = per(B) per(C)
    with 17 x 17 blocks, and by the rank-one closed form per(x y^T) = n! prod x prod y."""
    import math
    n, h = 34, 17
    g = np.random.default_rng(3434)
    b = (g.standard_normal((h, h)) + 1j * g.standard_normal((h, h))) / np.sqrt(2 * h)
    c = (g.standard_normal((h, h)) + 1j * g.standard_normal((h, h))) / np.sqrt(2 * h)
    blk = np.zeros((n, n), dtype=np.complex128)
    blk[:h, :h] = b
    blk[h:, h:] = c
    x = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
    y = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
    r1 = np.outer(x, y)
    with lp.Plan(n, "c128", method=lp.METHOD_SZ, max_batch=2, mem_budget_bytes=150 << 30) as p:
        assert p.describe()["sz_single_nmax"] == n
        got, st = lp.permanents([blk, r1], "c128", plan=p, return_status=True)
    assert list(st) == [lp.PERM_OK, lp.PERM_OK]
    want_blk = oracle_c(b) * oracle_c(c)
    scale_blk = oracle.per_abs(b) * oracle.per_abs(c)
    assert abs(got[0] - want_blk) <= 1e-12 * scale_blk, (got[0], want_blk)
    want_r1 = math.factorial(n) * np.prod(x) * np.prod(y)
    scale_r1 = math.factorial(n) * np.prod(np.abs(x)) * np.prod(np.abs(y))
    assert abs(got[1] - want_r1) <= 1e-12 * scale_r1, (got[1], want_r1)


@pytest.mark.parametrize("method", ["sz", "ryser"])
def test_compact_orders_general_matrices(lp, method):
    """General complex matrices of order 33 (and 34) from the serving stream -- the orders
    with compact Store-zechin tables -- against the oracle's stored double-double values
    (tests/golden/make_compact_orders.py)."""
    gold = _golden("compact_orders.json")
    reqs = wl.uneven_requests(**gold["stream"])
    assert gold["cases"] and gold["cases"][0]["n"] == 33
    m = lp.METHOD_SZ if method == "sz" else lp.METHOD_RYSER
    for c in gold["cases"]:
        a = reqs[c["index"]].mat
        assert a.shape == (c["n"], c["n"]) and reqs[c["index"]].dtype == "c128"
        with lp.Plan(c["n"], "c128", method=m, max_batch=1, mem_budget_bytes=100 << 30) as p:
            got = lp.permanents([a], "c128", plan=p)[0]
        want = complex(*c["per"])
        assert abs(got - want) <= 1e-12 * c["per_abs"], (c["n"], method, got, want)

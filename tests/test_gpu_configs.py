"""The five workloads end to end through the C ABI, against the oracle.

* 5-boson (all 126 patterns + 100 0/1): tests/test_gpu_parity.py.
* batched n = 20: the full 4096 + 4096 batch in the launch configuration the
  bench times (autotuned plan); a seeded sample of outputs against the oracle,
  every status OK.
* single n = 32: Store-zechin and Ryser against the stored oracle value.
* uneven n = 8..28: every n <= 22 against the oracle; larger n Store-zechin
  against GPU Ryser (bit-exact for integers; complex within 2e-12 per(|A|),
  per(|A|) taken from the GPU on |A|, which has no cancellation).
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


def test_uneven_sample(lp):
    reqs = wl.uneven_requests(count=160)
    for dt in ("c128", "u01"):
        mats = [r.mat for r in reqs if r.dtype == dt]
        res, st = lp.permanents(mats, dt, return_status=True)
        assert (np.asarray(st) == lp.PERM_OK).all()
        big = [i for i, m in enumerate(mats) if m.shape[0] > 22]
        ry = lp.permanents([mats[i] for i in big], dt, method=lp.METHOD_RYSER) if big else []
        for i, m in enumerate(mats):
            if m.shape[0] <= 22:
                if dt == "c128":
                    assert abs(res[i] - oracle_c(m)) <= tol_c(m)
                else:
                    assert res[i] == oracle_i(m)
        if dt == "c128" and big:
            scale = lp.permanents([np.abs(mats[i]).astype(np.complex128) for i in big], "c128")
            for k, i in enumerate(big):
                assert abs(res[i] - ry[k]) <= 2e-12 * abs(scale[k])
        elif big:
            assert [res[i] for i in big] == list(ry)


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


def test_store_zechin_n34_in_hbm(lp):
    """The largest Store-zechin order: n = 34 complex, 139 GB of chain tables in HBM
    (a 150 GB budget).  Pinned by the oracle through a block-diagonal matrix,
    per(B + C) = per(B) per(C) with 17 x 17 blocks, and by the rank-one closed form
    per(x y^T) = n! prod x prod y."""
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

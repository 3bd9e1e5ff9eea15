"""The dataflow form of the layer path (sz_flow_c128): one persistent launch in
which each chain starts once its predecessor chains are done, instead of one
launch per layer.  It must give the layer path's bits for every order up to 24
and every number of matrices, and the oracle's values."""
import numpy as np
import pytest

from tests.gpu_helpers import oracle_c, rand_complex, tol_c

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


@pytest.mark.parametrize("n", [6, 13, 16, 20, 21, 24])
@pytest.mark.parametrize("count", [1, 3])
def test_flow_same_bits_as_layers(lp, monkeypatch, n, count):
    mats = [rand_complex(n, 13000 + 10 * n + i) for i in range(count)]
    res = {}
    for flow in ("0", "1"):
        monkeypatch.setenv("LIBPERM_SZ_FLOW", flow)
        with lp.Plan(n, "c128", method=lp.METHOD_SZ, max_batch=count) as p:
            got, st = lp.permanents(mats, "c128", plan=p, return_status=True)
        assert list(st) == [lp.PERM_OK] * count
        res[flow] = list(got)
    assert res["1"] == res["0"]
    if n <= 21:
        assert abs(res["1"][0] - oracle_c(mats[0])) <= tol_c(mats[0])


def test_flow_mixed_orders_in_one_call(lp, monkeypatch):
    """Several orders in one call: each order's group is one dataflow launch, in turn."""
    monkeypatch.setenv("LIBPERM_SZ_FLOW", "1")
    ns = [22, 17, 22, 23, 14]
    mats = [rand_complex(n, 13500 + i) for i, n in enumerate(ns)]
    with lp.Plan(24, "c128", method=lp.METHOD_SZ, max_batch=len(mats)) as p:
        got = lp.permanents(mats, "c128", plan=p)
    for g, m in zip(got, mats):
        assert g == lp.permanents([m], "c128", method=lp.METHOD_SZ)[0]
    assert abs(got[1] - oracle_c(mats[1])) <= tol_c(mats[1])


@pytest.mark.parametrize("count", [1, 2, 4])
def test_flow_chain_width_by_order_and_count(lp, count):
    """At most four matrices of an order up to 24 take chains of 2^w, w = floor((n - 1 +
    floor(log2 count)) / 2) clamped to 9..12; the bits are those of any fixed width."""
    with lp.Plan(24, "c128", method=lp.METHOD_SZ) as p:
        d = p.describe()
        assert d["chain_width_layer_few_n20"] == 9 and d["chain_width_layer_few"] == 11
    for n in (12, 18, 23):
        mats = [rand_complex(n, 13700 + 10 * n + i) for i in range(count)]
        res = []
        for low in (0, 12):
            with lp.Plan(n, "c128", method=lp.METHOD_SZ, max_batch=count, low_cols=low) as p:
                got, st = lp.permanents(mats, "c128", plan=p, return_status=True)
            assert list(st) == [lp.PERM_OK] * count
            res.append(list(got))
        assert res[0] == res[1]
        if n <= 18:
            assert abs(res[0][0] - oracle_c(mats[0])) <= tol_c(mats[0])

"""One matrix's Ryser code range split over ranks, on one GPU.

Ranks are emulated one after another on the same GPU: each computes the
partial sums of its share of the pieces (perm_ryser_partials), the shares are
concatenated in rank order, and perm_ryser_finish sums them.  No rank waits on
another.  The result must be the same bits as perm_batch with Ryser for every
number of ranks, and within the oracle's tolerance (complex) or exact
(integers)."""
import json
import os

import numpy as np
import pytest

from tests.gpu_helpers import oracle_c, oracle_i, rand01, rand_complex, tol_c

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


def _split_on_one_gpu(lp, plan, a, dtype, world):
    from paper_1802_02779_gb300 import ryser_split
    n = a.shape[0]
    npdt = np.complex128 if dtype == "c128" else np.int64
    dev = torch.from_numpy(np.ascontiguousarray(a, dtype=npdt).reshape(-1)).cuda()
    pieces, pb = lp.ryser_pieces(n, dtype)
    parts = []
    for b, e in ryser_split.shares(pieces, world):
        buf = torch.empty(max(1, (e - b) * pb), dtype=torch.uint8, device="cuda")
        plan.ryser_partials(dev, n, b, e, buf)
        parts.append(buf[: (e - b) * pb])
    full = torch.cat(parts)
    assert full.numel() == pieces * pb
    words = plan.describe().get("out_words", 2)
    out = torch.empty(1, dtype=torch.complex128, device="cuda") if dtype == "c128" else \
        torch.empty(words, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    plan.ryser_finish(n, full, out, st)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return (complex(o[0]) if dtype == "c128" else lp.words_to_int(o)), int(st.item())


@pytest.mark.parametrize("n", [1, 9, 17, 18, 24])
def test_complex_split_same_bits_for_every_world(lp, n):
    a = rand_complex(n, 7000 + n)
    with lp.Plan(n, "c128", method=lp.METHOD_RYSER) as plan:
        ref = lp.permanents([a], "c128", plan=plan)[0]
        for world in (1, 2, 3, 4, 8):
            got, st = _split_on_one_gpu(lp, plan, a, "c128", world)
            assert st == lp.PERM_OK
            assert got == ref, (n, world, got, ref)
    assert abs(ref - oracle_c(a)) <= tol_c(a)


def test_complex_n28_split_against_stored_oracle(lp):
    from paper_1802_02779_gb300 import workloads as wl
    with open(os.path.join(os.path.dirname(__file__), "golden", "large_complex.json")) as f:
        gold = json.load(f)
    c = next(c for c in gold["cases"] if c["stream"] == "uneven" and c["n"] == 28)
    a = wl.uneven_requests(**gold["streams"]["uneven"])[c["index"]].mat
    with lp.Plan(28, "c128", method=lp.METHOD_RYSER) as plan:
        ref = lp.permanents([a], "c128", plan=plan)[0]
        got, st = _split_on_one_gpu(lp, plan, a, "c128", 4)
    assert st == lp.PERM_OK and got == ref
    assert abs(got - complex(*c["per"])) <= 1e-12 * c["per_abs"]


@pytest.mark.parametrize("n,dtype,kind", [(14, "u01", "bern"), (26, "u01", "bern"), (20, "i64", "small"),
                                          (18, "i64", "large"), (9, "i64", "small")])
def test_integer_split_same_bits_for_every_world(lp, n, dtype, kind):
    g = np.random.default_rng(8000 + n)
    if kind == "bern":
        a = rand01(n, 8000 + n, 0.6)
    elif kind == "small":
        a = g.integers(0, 3, size=(n, n)).astype(np.int64)     # Glynn walk (small row sums)
    else:
        a = (g.random((n, n)) < 0.5).astype(np.int64)          # one row sum above 32767:
        a[0, 0] = 40000                                         # the Eq. 4 walk
    with lp.Plan(n, dtype, method=lp.METHOD_RYSER) as plan:
        ref, rst = lp.permanents([a], dtype, plan=plan, return_status=True)
        for world in (1, 2, 3, 5):
            got, st = _split_on_one_gpu(lp, plan, a, dtype, world)
            assert st == int(rst[0])
            assert got == ref[0], (n, world)
    assert st == lp.PERM_OK
    assert ref[0] == oracle_i(a)


def test_wide_split_dense_n36(lp):
    """192-bit (PERM_FLAG_WIDE) 0/1 matrix of order 36: 2^19 pieces over 3 ranks."""
    n = 36
    a = np.ones((n, n), dtype=np.int64)
    for k in range(14):
        a[k, (3 * k + 1) % n] = 0
    with lp.Plan(n, "u01", method=lp.METHOD_RYSER, flags=lp.FLAG_WIDE) as plan:
        ref = lp.permanents([a], "u01", plan=plan)[0]
        got, st = _split_on_one_gpu(lp, plan, a, "u01", 3)
    assert st == lp.PERM_OK and got == ref and got > (1 << 128)


def test_module_entry_single_rank(lp):
    from paper_1802_02779_gb300 import ryser_split
    a = rand_complex(20, 7100)
    with lp.Plan(20, "c128", method=lp.METHOD_RYSER) as plan:
        ref = lp.permanents([a], "c128", plan=plan)[0]
        dev = torch.from_numpy(a.reshape(-1)).cuda()
        out, st = ryser_split.permanent(plan, dev, 20)
        torch.cuda.synchronize()
    assert int(st.item()) == lp.PERM_OK and complex(out.cpu().numpy()[0]) == ref

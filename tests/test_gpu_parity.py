"""GPU parity: the CUDA Store-zechin and Ryser kernels against the CPU oracle.

Complex results must satisfy |per_gpu - per_oracle| <= 1e-12 * per(|A|);
integer results must be bit-exact."""
import math

import numpy as np
import pytest

import oracle
from paper_1802_02779_gb300 import workloads as wl
from tests.gpu_helpers import oracle_c, oracle_i, rand01, rand_complex, tol_c

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


METHODS = ["sz", "ryser"]


def meth(lp, name):
    return {"sz": lp.METHOD_SZ, "ryser": lp.METHOD_RYSER, "auto": lp.METHOD_AUTO}[name]


# ---------------------------------------------------------------------------
# 5-boson workload: all 126 collision-free patterns + 100 0/1 matrices
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", METHODS)
def test_five_boson_complex(lp, method):
    cm, _ = wl.five_boson()
    got = lp.permanents(list(cm), "c128", method=meth(lp, method))
    for g, m in zip(got, cm):
        assert abs(g - oracle_c(m)) <= tol_c(m)


@pytest.mark.parametrize("method", METHODS)
def test_five_boson_01(lp, method):
    _, im = wl.five_boson()
    got = lp.permanents(list(im), "u01", method=meth(lp, method))
    assert got == [oracle_i(m) for m in im]


# ---------------------------------------------------------------------------
# every order, several tiles and ragged chains
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", METHODS)
def test_complex_orders_1_to_18(lp, method):
    mats = [rand_complex(n, 1000 + n) for n in range(1, 19)]
    got = lp.permanents(mats, "c128", method=meth(lp, method))
    for g, m in zip(got, mats):
        assert abs(g - oracle_c(m)) <= tol_c(m), (m.shape[0], g, oracle_c(m))


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n", [19, 20, 21])
def test_complex_high_columns(lp, method, n):
    """n > 13 exercises the high-column chains (t = n - 13 layers)."""
    mats = [rand_complex(n, 2000 + n + k) for k in range(2)]
    got = lp.permanents(mats, "c128", method=meth(lp, method))
    for g, m in zip(got, mats):
        assert abs(g - oracle_c(m)) <= tol_c(m)


@pytest.mark.parametrize("method", METHODS)
def test_01_orders_1_to_22(lp, method):
    mats = [rand01(n, 3000 + n, p=0.6) for n in range(1, 23)]
    got = lp.permanents(mats, "u01", method=meth(lp, method))
    assert got == [oracle_i(m) for m in mats]


@pytest.mark.parametrize("method", METHODS)
def test_small_integers(lp, method):
    g = np.random.default_rng(5)
    mats = [g.integers(0, 6, size=(n, n)).astype(np.int64) for n in (2, 5, 9, 14, 17)]
    got = lp.permanents(mats, "i64", method=meth(lp, method))
    assert got == [oracle_i(m) for m in mats]


# ---------------------------------------------------------------------------
# closed forms and 128-bit integers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("n", [20, 21, 23])
def test_ones_and_derangements_u128(lp, method, n):
    J = np.ones((n, n), dtype=np.int64)
    D = J - np.eye(n, dtype=np.int64)
    got = lp.permanents([J, D], "u01", method=meth(lp, method))
    d = [1, 0]
    for k in range(2, n + 1):
        d.append((k - 1) * (d[-1] + d[-2]))
    assert got == [math.factorial(n), d[n]]


@pytest.mark.parametrize("method", METHODS)
def test_rank_one_complex_closed_form(lp, method):
    for n in (9, 17, 22):
        g = np.random.default_rng(40 + n)
        x = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
        y = (g.standard_normal(n) + 1j * g.standard_normal(n)) / 2
        want = math.factorial(n) * np.prod(x) * np.prod(y)
        scale = math.factorial(n) * np.prod(np.abs(x)) * np.prod(np.abs(y))
        got = lp.permanents([np.outer(x, y)], "c128", method=meth(lp, method))[0]
        assert abs(got - want) <= 1e-12 * scale, (n, got, want)


def test_empty_and_one(lp):
    got = lp.permanents([np.zeros((0, 0), np.complex128), np.array([[2 - 1j]])], "c128")
    assert got[0] == 1 and got[1] == 2 - 1j
    got = lp.permanents([np.zeros((0, 0), np.int64), np.array([[1]])], "u01")
    assert got == [1, 1]


def test_item_status_overflow_and_invalid(lp):
    big = np.full((4, 4), 1 << 40, dtype=np.int64)          # bound (2^42)^4 = 2^168
    neg = np.array([[1, -1], [2, 3]], dtype=np.int64)
    ok = np.array([[1, 2], [3, 4]], dtype=np.int64)
    res, st = lp.permanents([big, neg, ok], "i64", return_status=True)
    assert list(st) == [lp.PERM_EOVERFLOW, lp.PERM_EINVAL, lp.PERM_OK]
    assert res[2] == 10
    two = np.array([[1, 2], [0, 1]], dtype=np.int64)
    _, st = lp.permanents([two], "u01", return_status=True)
    assert list(st) == [lp.PERM_EINVAL]


# ---------------------------------------------------------------------------
# determinism: alone vs batched vs plain launches, bit for bit
# ---------------------------------------------------------------------------
def test_alone_vs_mix_bitwise(lp):
    mats = [rand_complex(n, 7000 + n) for n in (5, 12, 16, 20, 14, 3, 20, 9)]
    mixed = lp.permanents(mats, "c128")
    for i, m in enumerate(mats):
        alone = lp.permanents([m], "c128")[0]
        assert alone == mixed[i]
    plain = lp.permanents(mats, "c128", flags=lp.FLAG_PLAIN)
    assert list(plain) == list(mixed)


def test_batched_kernel_and_layer_path_same_bits(lp):
    """A call with at least as many Store-zechin matrices as SMs runs the batched
    kernel (one CTA per matrix, chain width 12); one matrix alone runs the layer
    path (the chains of each layer over the whole GPU, chain width 13).  Every
    entry is summed over its columns in ascending order on both, so the bits agree."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ns = [16, 20, 9, 13, 18] * ((sms + 4) // 5 + 1)
    mats = [rand_complex(n, 9300 + i) for i, n in enumerate(ns)]
    batched = lp.permanents(mats, "c128")
    for i in range(0, len(mats), 37):          # a sample, one matrix per call
        assert lp.permanents([mats[i]], "c128")[0] == batched[i]
    for i in (0, 1, 4):
        assert abs(batched[i] - oracle_c(mats[i])) <= tol_c(mats[i])


def test_sz_and_ryser_agree_n24(lp):
    m = rand_complex(24, 99)
    a = lp.permanents([m], "c128", method=lp.METHOD_SZ)[0]
    b = lp.permanents([m], "c128", method=lp.METHOD_RYSER)[0]
    scale = oracle.per_abs(m)
    assert abs(a - b) <= 2e-12 * scale


# ---------------------------------------------------------------------------
# CUDA-graph replay (PERM_FLAG_GRAPH): same bits as direct launches, and a
# replay reads the buffers' current contents
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["auto", "ryser"])
def test_graph_replay(lp, method):
    sizes = [0, 6, 12, 20, 23, 14, 20, 9]
    mats = [rand_complex(n, 8100 + i) for i, n in enumerate(sizes)]
    flat = np.concatenate([m.reshape(-1) for m in mats])
    dev = torch.from_numpy(flat).cuda()
    s = torch.cuda.Stream()
    outs = {}
    for flags in (0, lp.FLAG_GRAPH):
        with lp.Plan(max(sizes), "c128", method=meth(lp, method), flags=flags) as p:
            out = torch.empty(len(sizes), dtype=torch.complex128, device="cuda")
            st = torch.empty(len(sizes), dtype=torch.int32, device="cuda")
            res = []
            for rep in range(3):
                with torch.cuda.stream(s):
                    p.batch(dev, sizes, out, st, s)
                s.synchronize()
                res.append(out.cpu().numpy().copy())
                assert int(st.abs().sum()) == 0
            assert (res[0] == res[1]).all() and (res[1] == res[2]).all()
            # new contents, same buffers: scale matrix 3 (n = 20) by 2 -> per times 2^20
            dev2 = dev.clone()
            o3 = sum(n * n for n in sizes[:3])
            dev.view(-1)[o3:o3 + 20 * 20] *= 2
            with torch.cuda.stream(s):
                p.batch(dev, sizes, out, st, s)
            s.synchronize()
            scaled = out.cpu().numpy().copy()
            dev.copy_(dev2)
            outs[flags] = (res[0], scaled)
    assert (outs[0][0] == outs[lp.FLAG_GRAPH][0]).all()
    assert (outs[0][1] == outs[lp.FLAG_GRAPH][1]).all()
    assert outs[0][1][3] == outs[0][0][3] * 2 ** 20


# ---------------------------------------------------------------------------
# autotuner: picks a CTA size / chain width, results stay bit-identical
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["c128", "u01"])
def test_autotuned_plan_same_bits(lp, dtype):
    n = 16
    mats = [rand_complex(n, 9100 + k) if dtype == "c128" else rand01(n, 9100 + k) for k in range(40)]
    # integer plans use Store-zechin (and so the tuner) only when it is asked for
    method = lp.METHOD_AUTO if dtype == "c128" else lp.METHOD_SZ
    with lp.Plan(n, dtype, method=method, flags=lp.FLAG_AUTOTUNE) as pt:
        d = pt.describe()
        assert d["autotuned"] is True
        assert d["chain_width_batched"] in (11, 12, 13)
        tuned = lp.permanents(mats, dtype, plan=pt)
    plain = lp.permanents(mats, dtype)
    if dtype == "c128":
        assert list(tuned) == list(plain)
    else:
        assert tuned == plain


def test_autotuned_crossover_and_layer_shape_same_bits(lp, tmp_path, monkeypatch):
    """A complex plan of n_max = 24 tunes the batched kernel, the batched/layer
    crossover (19..22) and the layer path's CTA size, chain width and grid; every
    tuned choice is reported by perm_plan_describe, kept in LIBPERM_TUNE_CACHE, and
    gives the default plan's bits on a batch that takes both paths."""
    monkeypatch.setenv("LIBPERM_TUNE_CACHE", str(tmp_path / "tune.txt"))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ns = [16, 19, 20, 21, 22, 24] * ((sms + 5) // 6 + 1)
    mats = [rand_complex(n, 9500 + i) for i, n in enumerate(ns)]
    with lp.Plan(24, "c128", flags=lp.FLAG_AUTOTUNE, max_batch=len(mats)) as pt:
        d = pt.describe()
        assert d["autotuned"] is True
        assert 18 <= d["sz_batch_nmax"] <= 22
        assert (d["layer_cta_threads_small"], d["chain_width_layer_small"]) in ((512, 13), (384, 12), (512, 12))
        assert d["layer_ctas_per_sm_small"] in (1, 2, 4)
        assert (d["layer_cta_threads"], d["chain_width_single"]) == (768, 13)
        tuned = lp.permanents(mats, "c128", plan=pt)
    assert "perm-tune2" in (tmp_path / "tune.txt").read_text()
    with lp.Plan(24, "c128", max_batch=len(mats)) as p0:
        plain = lp.permanents(mats, "c128", plan=p0)
    assert list(tuned) == list(plain)
    for i in (0, 3, 5):
        assert abs(tuned[i] - oracle_c(mats[i])) <= tol_c(mats[i])


# ---------------------------------------------------------------------------
# all collision-free patterns in one pass (perm_patterns)
# ---------------------------------------------------------------------------
def test_patterns_five_boson(lp):
    """rows 0..4 of the 9x9 Haar unitary: one 5x9 pass gives all 126 amplitudes,
    bit-identical to the 126 separate 5x5 permanents."""
    u = wl.haar_unitary(9, 18021)
    got = lp.patterns(u[:5])[0]
    subs = lp.colex_subsets(9, 5)
    assert len(got) == 126
    sep = lp.permanents([np.ascontiguousarray(u[:5][:, list(c)]) for c in subs], "c128")
    assert list(got) == list(sep)
    for c, g in zip(subs[:20], got[:20]):
        m = np.ascontiguousarray(u[:5][:, list(c)])
        assert abs(g - oracle_c(m)) <= tol_c(m)


@pytest.mark.parametrize("rows,cols", [(1, 4), (3, 3), (4, 11), (6, 13)])
def test_patterns_shapes(lp, rows, cols):
    g = np.random.default_rng(rows * 100 + cols)
    mats = (g.standard_normal((3, rows, cols)) + 1j * g.standard_normal((3, rows, cols))) / np.sqrt(2 * cols)
    got = lp.patterns(mats)
    subs = lp.colex_subsets(cols, rows)
    for i in range(3):
        sep = lp.permanents([np.ascontiguousarray(mats[i][:, list(c)]) for c in subs], "c128")
        assert list(got[i]) == list(sep)


def test_patterns_with_collisions_sum_rule(lp):
    """All 1287 outputs of 5 photons in 9 modes (collisions included) in one pass:
    the probabilities |per|^2 / prod t_j! sum to 1 (a unitary), each amplitude
    matches the oracle, and the collision-free ones match perm_patterns."""
    import math
    u = wl.haar_unitary(9, 18021)
    amps = lp.patterns_multiset(u[:5])[0]
    occ = lp.colex_multisets(9, 5)
    assert len(amps) == len(occ) == 1287
    total = sum(abs(a) ** 2 / np.prod([math.factorial(t) for t in o]) for a, o in zip(amps, occ))
    assert abs(total - 1.0) < 1e-12
    for idx in np.random.default_rng(9).choice(len(occ), size=40, replace=False):
        cols = [j for j, t in enumerate(occ[idx]) for _ in range(t)]
        m = np.ascontiguousarray(u[:5][:, cols])
        assert abs(amps[idx] - oracle_c(m)) <= tol_c(m)
    free = lp.patterns(u[:5])[0]
    free_occ = [tuple(1 if j in c else 0 for j in range(9)) for c in lp.colex_subsets(9, 5)]
    lookup = dict(zip(occ, amps))
    for o, f in zip(free_occ, free):
        assert abs(lookup[o] - f) <= 1e-14


def test_patterns_multiset_limits(lp):
    big = np.zeros((6, 13), dtype=np.complex128)      # C(18, 6) = 18564 > 6000
    with pytest.raises(lp.LibpermError):
        lp.patterns_multiset(big)

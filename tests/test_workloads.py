"""The seeded workload generators: deterministic, and with the shapes, sizes and
mixes the benchmark and tests state (5-boson, batched n = 20, single n = 32,
uneven n = 8..28, Poisson serving n = 10..36)."""
import itertools

import numpy as np

from paper_1802_02779_gb300 import workloads as wl


def test_five_boson_patterns_and_bernoulli():
    cm, im = wl.five_boson()
    assert cm.shape == (126, 5, 5) and cm.dtype == np.complex128
    assert im.shape == (100, 5, 5) and im.dtype == np.int64
    assert set(np.unique(im)) <= {0, 1}
    u = wl.haar_unitary(9, wl.SEED_BASE + 1)
    subs = list(itertools.combinations(range(9), 5))
    for k in (0, 57, 125):                       # lexicographic column subsets of rows 0..4
        assert np.array_equal(cm[k], u[:5][:, list(subs[k])])


def test_batched_n20_is_deterministic_and_shaped():
    a_c, a_i = wl.batched_n20(count=16)
    b_c, b_i = wl.batched_n20(count=16)
    assert np.array_equal(a_c, b_c) and np.array_equal(a_i, b_i)
    assert a_c.shape == (16, 20, 20) and a_i.shape == (16, 20, 20)
    # complex: rows 0..19 of one Haar unitary -> every row of a submatrix has norm <= 1
    assert np.all(np.linalg.norm(a_c, axis=2) <= 1.0 + 1e-12)
    assert 0.4 < a_i.mean() < 0.6


def test_single_n32_scale():
    a = wl.single_n32()
    assert a.shape == (32, 32) and a.dtype == np.complex128
    # entries ~ CN(0, 1) / 32: mean |z|^2 close to 1 / 1024
    assert abs(np.mean(np.abs(a) ** 2) * 1024 - 1.0) < 0.15
    assert np.array_equal(a, wl.single_n32())


def test_uneven_requests_mix():
    reqs = wl.uneven_requests(count=2000)
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 8 and ns.max() <= 28 and len(set(ns)) == 21
    frac_c = np.mean([r.dtype == "c128" for r in reqs])
    assert 0.66 < frac_c < 0.74
    for r in reqs[:50]:
        assert r.mat.shape == (r.n, r.n)
        if r.dtype == "u01":
            assert r.mat.dtype == np.int64 and set(np.unique(r.mat)) <= {0, 1}
    again = wl.uneven_requests(count=2000)
    assert all(np.array_equal(x.mat, y.mat) for x, y in zip(reqs[:20], again[:20]))


def test_poisson_arrivals_rate():
    reqs = wl.poisson_arrivals(count=4000, rate_per_s=2.0)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] - 2.0) < 0.15         # arrivals per second
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 10 and ns.max() <= 36

"""The continuous-batching server: results, alone-vs-mix equality, error paths."""
import ctypes
import os
import subprocess
import sys
import time

import numpy as np
import pytest

from tests.gpu_helpers import oracle_c, oracle_i, rand01, rand_complex, tol_c

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lp():
    assert torch.cuda.is_available()
    from paper_1802_02779_gb300 import build
    build.build()
    from paper_1802_02779_gb300 import libperm
    libperm.load()
    return libperm


def make_requests():
    reqs = []
    g = np.random.default_rng(77)
    for k in range(60):
        n = int(g.integers(3, 25))
        if k % 3 == 2:
            reqs.append(("u01", rand01(n, 500 + k, p=float(g.uniform(0.3, 0.7)))))
        else:
            reqs.append(("c128", rand_complex(n, 600 + k)))
    reqs.append(("i64", g.integers(0, 4, size=(7, 7)).astype(np.int64)))
    return reqs


def test_server_matches_alone_and_oracle(lp):
    reqs = make_requests()
    with lp.Server(mem_budget_bytes=2 << 30) as srv:
        tickets = []
        for i, (dt, m) in enumerate(reqs):
            tickets.append(srv.submit(m, dt))
            if i % 7 == 0:
                time.sleep(0.002)          # let batches start while others arrive
        results = srv.wait_all(tickets, timeout_s=300)
    for (dt, m), (val, st) in zip(reqs, results):
        assert st == lp.PERM_OK
        alone = lp.permanents([m], dt)[0]
        if dt == "c128":
            assert abs(val - oracle_c(m)) <= tol_c(m)
            # same method and order for n within the batch lane and the table budget
            assert val == alone, (m.shape[0], val, alone)
        else:
            assert val == oracle_i(m) == alone


def test_server_large_lane_ryser_fallback(lp):
    """A request whose Store-zechin tables exceed the table budget runs with Ryser."""
    m = rand_complex(23, 901)
    with lp.Server(mem_budget_bytes=64 << 20) as srv:   # 23 needs ~91 MB of chains
        t = srv.submit(m, "c128")
        (val, st), = srv.wait_all([t], timeout_s=300)
    assert st == lp.PERM_OK
    assert abs(val - oracle_c(m)) <= tol_c(m)


def test_unknown_ticket_and_queue_full(lp):
    with lp.Server(mem_budget_bytes=1 << 30, max_batch=2) as srv:
        assert srv.poll(123456789) == ("missing", None)
        m = rand_complex(18, 3)
        saw_again = False
        tickets = []
        for _ in range(5000):
            ok, t = srv.try_submit(m, "c128")
            if not ok:
                saw_again = True
                break
            tickets.append(t)
        assert saw_again
        srv.wait_all(tickets, timeout_s=300)


def test_destroy_times_out_with_work_in_flight():
    """perm_server_destroy returns PERM_ETIMEDOUT when in-flight work outlives the
    timeout (run in a child process: the timed-out server is left to drain)."""
    code = r'''
import numpy as np, sys
sys.path.insert(0, %r)
from paper_1802_02779_gb300 import libperm as lp
srv = lp.Server(mem_budget_bytes=1 << 30)
a = (np.random.default_rng(1).standard_normal((30, 30)) + 0j) / 30
for _ in range(4):
    srv.submit(a, "c128")
rc = srv.destroy(timeout_ms=0)
print("RC", rc)
''' % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    from paper_1802_02779_gb300 import libperm as lp
    assert f"RC {lp.PERM_ETIMEDOUT}" in r.stdout


def _uneven_large_complex(lp, orders):
    """Large complex requests of the uneven stream with their stored oracle values."""
    import json
    from paper_1802_02779_gb300 import workloads as wl
    with open(os.path.join(ROOT, "tests", "golden", "large_complex.json")) as f:
        gold = json.load(f)
    reqs = wl.uneven_requests(**gold["streams"]["uneven"])
    cases = [c for c in gold["cases"] if c["stream"] == "uneven" and c["n"] in orders]
    return [(reqs[c["index"]].mat, complex(*c["per"]), c["per_abs"]) for c in cases]


@pytest.mark.parametrize("budget_mb", [8192, 700])
def test_table_lane_concurrent_jobs_same_bits_as_alone(lp, budget_mb):
    """Large complex requests of orders 23..26 submitted together: with an 8 GB
    budget several table jobs are in flight at once (same-order requests share
    layer launches); with 700 MB one order-26 job (675 MB of tables) fits at a
    time and the others wait for its memory.  Every result is the bits
    perm_batch gives the matrix alone and within the oracle's tolerance."""
    cases = _uneven_large_complex(lp, (23, 24, 25, 26))
    assert len(cases) >= 20
    with lp.Server(mem_budget_bytes=budget_mb << 20) as srv:
        tickets = [srv.submit(a, "c128") for a, _, _ in cases]
        res = srv.wait_all(tickets, timeout_s=600)
    for (a, want, scale), (val, st) in zip(cases, res):
        assert st == lp.PERM_OK
        alone = lp.permanents([a], "c128")[0]
        assert val == alone, (a.shape[0], val, alone)
        assert abs(val - want) <= 1e-12 * scale

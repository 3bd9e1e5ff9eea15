"""Write tests/golden/large_complex.json: the oracle's permanents of seeded
complex workload matrices of order 23..31, with per(|A|) for the tolerance.

The matrices are Haar-unitary submatrices drawn by the input generators:
  * the uneven-size stream (workloads.uneven_requests(count=200)): every
    complex request of order n = 23..28 (43 matrices);
  * the serving stream's requests (workloads.uneven_requests(count=300,
    seed=SEED_BASE + 8, n_lo=10, n_hi=36), the matrices poisson_arrivals
    draws): the first complex request of each order n = 29..31.
Both values come from the double-double Ryser oracle (Eq. 4 over all 2^n
column subsets).  Calls only oracle/ and the input generators; about half an
hour on eight cores.  Run:  python tests/golden/make_large_complex.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1802_02779_gb300 import workloads as wl  # noqa: E402

# (stream name, generator keyword arguments, orders, matrices per order (None: all))
STREAMS = [
    ("uneven", dict(count=200), range(23, 29), None),
    ("serving", dict(count=300, seed=wl.SEED_BASE + 8, n_lo=10, n_hi=36), range(29, 32), 1),
]


def stream_requests(name):
    for s, kw, _, _ in STREAMS:
        if s == name:
            return wl.uneven_requests(**kw)
    raise KeyError(name)


def selected():
    """[(stream, index, n)] in a fixed order."""
    out = []
    for name, kw, orders, per_n in STREAMS:
        reqs = wl.uneven_requests(**kw)
        for n in orders:
            idx = [i for i, r in enumerate(reqs) if r.dtype == "c128" and r.n == n][:per_n]
            out += [(name, i, n) for i in idx]
    return out


def main():
    cases = []
    cache = {}
    for name, i, n in selected():
        if name not in cache:
            cache[name] = stream_requests(name)
        a = cache[name][i].mat
        t0 = time.time()
        r = oracle.per_ryser(a)
        rabs = oracle.per_ryser(np.abs(a).astype(np.complex128))
        cases.append({"stream": name, "index": i, "n": n, "per_dd": list(r),
                      "per": [r[0] + r[1], r[2] + r[3]], "per_abs": rabs[0] + rabs[1],
                      "oracle_seconds": time.time() - t0})
        print(name, i, n, cases[-1]["per"], cases[-1]["per_abs"], f"{time.time() - t0:.1f}s", flush=True)
    out = {
        "_what": "per(A) and per(|A|) of complex workload matrices of order 23..31 by the "
                 "double-double Ryser oracle (Eq. 4); written by tests/golden/make_large_complex.py",
        "streams": {name: kw for name, kw, _, _ in STREAMS},
        "threads": oracle.max_threads(),
        "cases": cases,
    }
    with open(os.path.join(HERE, "large_complex.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

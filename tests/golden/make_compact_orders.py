"""Write tests/golden/compact_orders.json: the oracle's permanents of the first
complex request of order 33 and of order 34 in the serving stream's requests
(workloads.uneven_requests(count=300, seed=SEED_BASE + 8, n_lo=10, n_hi=36),
the matrices poisson_arrivals draws), with per(|A|) for the tolerance.  These
orders keep compact Store-zechin tables on the GPU.

Both values come from the double-double Ryser oracle (Eq. 4 over all 2^n column
subsets).  Calls only oracle/ and the input generators; about three hours on
eight cores.  Run:  python tests/golden/make_compact_orders.py
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

STREAM = dict(count=300, seed=wl.SEED_BASE + 8, n_lo=10, n_hi=36)
ORDERS = (33, 34)


def selected():
    """[(index, n)]: the first complex request of each order in ORDERS."""
    reqs = wl.uneven_requests(**STREAM)
    return [(next(i for i, r in enumerate(reqs) if r.dtype == "c128" and r.n == n), n) for n in ORDERS]


def main():
    reqs = wl.uneven_requests(**STREAM)
    cases = []
    for i, n in selected():
        a = reqs[i].mat
        t0 = time.time()
        r = oracle.per_ryser(a)
        rabs = oracle.per_ryser(np.abs(a).astype(np.complex128))
        cases.append({"index": i, "n": n, "per_dd": list(r), "per": [r[0] + r[1], r[2] + r[3]],
                      "per_abs": rabs[0] + rabs[1], "oracle_seconds": time.time() - t0})
        print(i, n, cases[-1]["per"], cases[-1]["per_abs"], f"{time.time() - t0:.1f}s", flush=True)
        out = {
            "_what": "per(A) and per(|A|) of the first complex serving-stream requests of order 33 and 34 "
                     "by the double-double Ryser oracle (Eq. 4); written by tests/golden/make_compact_orders.py",
            "stream": STREAM,
            "threads": oracle.max_threads(),
            "cases": cases,
        }
        with open(os.path.join(HERE, "compact_orders.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

"""Write tests/golden/large_u01.json: the oracle's exact permanents of the 0/1
requests of order 23..28 in the seeded uneven-size stream
(workloads.uneven_requests(count=200)), every one of them.

The values come from the exact integer Ryser oracle (Eq. 4 over all 2^n
column subsets, modulo 2^256, far above any of these permanents).  Calls only
oracle/ and the input generators; a few minutes on eight cores.
Run:  python tests/golden/make_large_u01.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1802_02779_gb300 import workloads as wl  # noqa: E402

STREAM = dict(count=200)
ORDERS = range(23, 29)


def selected():
    """[(index, n)] of the 0/1 requests of order 23..28, in stream order."""
    reqs = wl.uneven_requests(**STREAM)
    return [(i, r.n) for i, r in enumerate(reqs) if r.dtype == "u01" and r.n in ORDERS]


def main():
    reqs = wl.uneven_requests(**STREAM)
    cases = []
    for i, n in selected():
        t0 = time.time()
        v = oracle.per_ryser(reqs[i].mat)
        cases.append({"index": i, "n": n, "per": str(v), "oracle_seconds": time.time() - t0})
        print(i, n, v, f"{time.time() - t0:.1f}s", flush=True)
    out = {
        "_what": "exact per(A) of the 0/1 requests of order 23..28 of "
                 "workloads.uneven_requests(count=200) by the exact integer Ryser oracle (Eq. 4); "
                 "written by tests/golden/make_large_u01.py",
        "stream": STREAM,
        "threads": oracle.max_threads(),
        "cases": cases,
    }
    with open(os.path.join(HERE, "large_u01.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

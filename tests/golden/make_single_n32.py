"""Write tests/golden/single_n32.json: the oracle's permanent of the seeded
single n = 32 workload matrix (i.i.d. complex Gaussian scaled by 1/32, seed
18025) and per(|A|), both by the double-double Ryser oracle (Eq. 4).

Calls only oracle/ (and the input generator).  Takes several minutes per
value on a few cores; run:  python tests/golden/make_single_n32.py
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


def main():
    a = wl.single_n32()
    t0 = time.time()
    r = oracle.per_ryser(a)
    t1 = time.time()
    rabs = oracle.per_ryser(np.abs(a).astype(np.complex128))
    t2 = time.time()
    out = {
        "_what": "per(A) and per(|A|) of workloads.single_n32() (n = 32, seed 18025, scale 1/32) "
                 "by the double-double Ryser oracle (Eq. 4); written by tests/golden/make_single_n32.py",
        "n": 32,
        "per_dd": list(r),
        "per": [r[0] + r[1], r[2] + r[3]],
        "per_abs": rabs[0] + rabs[1],
        "oracle_seconds": [t1 - t0, t2 - t1],
        "threads": oracle.max_threads(),
    }
    with open(os.path.join(HERE, "single_n32.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

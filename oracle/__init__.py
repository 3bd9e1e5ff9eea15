"""CPU oracle for matrix permanents (Su & Zheng, arXiv:1802.02779).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1802_02779_gb300``) never imports it and shares no code with it.

Contents
--------
* ``per_brute``     -- Eq. (1), Section 3.1: the sum over all n! permutations
                        (n <= 10), exact mod 2^256 for integers, double-double
                        for complex.
* ``per_ryser``     -- Eq. (4), Section 3.3: inclusion-exclusion over all 2^n
                        column subsets, exact mod 2^256 for integers,
                        double-double for complex; OpenMP over subset chunks.
* ``per_abs``       -- per(|A|), the scale of the complex tolerance.
* ``store_zechin``  -- the paper's Section 4 development with stored
                        sub-permanents, instrumented to count x and + (pins
                        Tables 1-4) and reference multiplicities (Section 4.2/4.3).
* ``cost_model``    -- Section 5.2: running times from operation counts and the
                        ENIAC/TRADIC rates (Table 5).

The C part (``perm_oracle.c``) is compiled by :func:`build` with gcc; nothing
here touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "perm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, out_path: str = None, defines=()) -> str:
    """Compile ``perm_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP).

    ``defines``/``out_path`` are used only by the planted-mistake test, which
    builds deliberately wrong variants into a temporary directory.
    """
    path = out_path or _LIB_PATH
    if (not force and not defines and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", *[f"-D{d}" for d in defines], _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _configure(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_per_brute_c128.argtypes = [ctypes.c_int, dp, dp]
    lib.oracle_per_brute_i64.argtypes = [ctypes.c_int, i64p, u64p]
    lib.oracle_per_ryser_c128.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
    lib.oracle_per_ryser_i64.argtypes = [ctypes.c_int, i64p, u64p, ctypes.c_int]
    lib.oracle_dd_add.argtypes = [dp, dp, dp]
    lib.oracle_dd_mul.argtypes = [dp, dp, dp]
    for f in ("oracle_per_brute_c128", "oracle_per_brute_i64",
              "oracle_per_ryser_c128", "oracle_per_ryser_i64"):
        getattr(lib, f).restype = ctypes.c_int
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _swap_library(lib):
    """Replace the loaded library (planted-mistake test only); returns the old one."""
    global _lib
    with _lock:
        old, _lib = _lib, lib
    return old


def max_threads() -> int:
    """OpenMP threads the Ryser oracle uses by default."""
    return int(_load().oracle_max_threads())


def _limbs_to_int(limbs) -> int:
    v = 0
    for i, w in enumerate(limbs):
        v |= int(w) << (64 * i)
    if v >> 255:            # two's complement, 256 bits
        v -= 1 << 256
    return v


def _as_square(a):
    a = np.asarray(a)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected a square matrix")
    return a


def _is_complex(a) -> bool:
    return np.iscomplexobj(a) or a.dtype.kind == "f"


def _call_int(fn, a, *extra):
    n = a.shape[0]
    buf = np.ascontiguousarray(a, dtype=np.int64)
    out = (ctypes.c_uint64 * 4)()
    rc = fn(n, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), out, *extra)
    if rc != 0:
        raise ValueError(f"oracle rejected the input (n={n})")
    return _limbs_to_int(out)


def _call_c128(fn, a, *extra):
    n = a.shape[0]
    buf = np.ascontiguousarray(a, dtype=np.complex128)
    out = (ctypes.c_double * 4)()
    rc = fn(n, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out, *extra)
    if rc != 0:
        raise ValueError(f"oracle rejected the input (n={n})")
    return (out[0], out[1], out[2], out[3])


def per_brute(a):
    """Eq. (1): sum over S_n of prod_i a[i, s(i)] (n <= 10).

    Integer input -> exact Python int.  Complex/real input -> ``DD`` result
    ``(re_hi, re_lo, im_hi, im_lo)``; use :func:`dd_to_complex` to round.
    """
    a = _as_square(a)
    lib = _load()
    if _is_complex(a):
        return _call_c128(lib.oracle_per_brute_c128, a)
    return _call_int(lib.oracle_per_brute_i64, a)


def per_ryser(a, threads: int = 0):
    """Eq. (4): (-1)^n sum_S (-1)^|S| prod_i sum_{j in S} a[i, j], all 2^n subsets.

    Integer input -> exact Python int (mod 2^256, signed).  Complex/real input
    -> double-double ``(re_hi, re_lo, im_hi, im_lo)``.  ``threads=0`` uses all
    OpenMP threads.
    """
    a = _as_square(a)
    lib = _load()
    if _is_complex(a):
        return _call_c128(lib.oracle_per_ryser_c128, a, int(threads))
    return _call_int(lib.oracle_per_ryser_i64, a, int(threads))


def dd_to_complex(r) -> complex:
    """Round a double-double complex result to the nearest complex128."""
    return complex(r[0] + r[1], r[2] + r[3])


def per(a, threads: int = 0):
    """per(A): brute force for n <= 8, Ryser above; complex results rounded."""
    a = _as_square(a)
    r = per_brute(a) if a.shape[0] <= 8 else per_ryser(a, threads)
    return dd_to_complex(r) if isinstance(r, tuple) else r


def per_abs(a, threads: int = 0) -> float:
    """per(|A|) for a complex matrix: the scale the tolerance is measured in."""
    a = _as_square(a)
    r = per(np.abs(a).astype(np.complex128), threads)
    return abs(r)


def dd_add(a, b):
    """Expose the oracle's double-double addition (for the primitive pins)."""
    lib = _load()
    x = (ctypes.c_double * 2)(*a)
    y = (ctypes.c_double * 2)(*b)
    o = (ctypes.c_double * 2)()
    lib.oracle_dd_add(x, y, o)
    return (o[0], o[1])


def dd_mul(a, b):
    """Expose the oracle's double-double multiplication (for the primitive pins)."""
    lib = _load()
    x = (ctypes.c_double * 2)(*a)
    y = (ctypes.c_double * 2)(*b)
    o = (ctypes.c_double * 2)()
    lib.oracle_dd_mul(x, y, o)
    return (o[0], o[1])

"""Python binding of libperm (ctypes): argument marshalling only.

Every permanent is computed by the CUDA kernels of ``libperm.so``; this module
only converts arguments.  PyTorch supplies device memory and streams.  There is
no CPU fallback: if ``libperm.so`` is missing or cannot be loaded, importing
this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libperm.so")

# perm_status
PERM_OK, PERM_EINVAL, PERM_ENOMEM, PERM_EOVERFLOW, PERM_ECUDA = 0, 1, 2, 3, 4
PERM_EAGAIN, PERM_ETIMEDOUT, PERM_ESHUTDOWN, PERM_ENOTFOUND = 5, 6, 7, 8
# perm_dtype
PERM_C128, PERM_U01, PERM_I64 = 1, 2, 3
# perm_method
METHOD_AUTO, METHOD_SZ, METHOD_RYSER = 0, 1, 2
FLAG_PLAIN = 1
FLAG_GRAPH = 2
FLAG_AUTOTUNE = 4
FLAG_WIDE = 8      # integer results as four uint64 words (256-bit slots), exact below 2^192

DTYPES = {"c128": PERM_C128, "u01": PERM_U01, "i64": PERM_I64}


class LibpermError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class PermOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t),
                ("max_batch", ctypes.c_int),
                ("method", ctypes.c_int),
                ("flags", ctypes.c_uint),
                ("ctas_per_sm", ctypes.c_int),
                ("low_cols", ctypes.c_int)]


# Every symbol include/libperm.h declares, with its ctypes signature.
_VP = ctypes.c_void_p
_SIGS = {
    "perm_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(PermOpts), ctypes.POINTER(_VP)]),
    "perm_plan_destroy": (ctypes.c_int, [_VP]),
    "perm_plan_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "perm_plan_describe": (ctypes.c_int, [_VP, ctypes.c_char_p, ctypes.c_size_t]),
    "perm_batch": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP, _VP, _VP]),
    "perm_batch_host": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP, _VP, _VP]),
    "perm_server_create": (ctypes.c_int, [ctypes.POINTER(PermOpts), _VP, ctypes.POINTER(_VP)]),
    "perm_submit": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "perm_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, _VP, ctypes.POINTER(ctypes.c_int)]),
    "perm_server_destroy": (ctypes.c_int, [_VP, ctypes.c_int]),
    "perm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "perm_version": (ctypes.c_char_p, []),
    "perm_measure_fp64_peak": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "perm_sz_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "perm_patterns": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "perm_patterns_multiset": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "perm_ryser_pieces": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_size_t)]),
    "perm_ryser_split": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "perm_ryser_partials": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, _VP, _VP]),
    "perm_ryser_finish": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
}

_lib = None


def load():
    """Load libperm.so (raises OSError/RuntimeError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libperm.so not built at {LIB_PATH}; run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def strerror(status: int) -> str:
    return load().perm_strerror(int(status)).decode()


def version() -> str:
    return load().perm_version().decode()


def _check(rc: int, where: str):
    if rc != PERM_OK:
        raise LibpermError(rc, where)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def measure_fp64_peak(ms_target: float = 200.0) -> float:
    """Sustained FP64 FMA throughput of the current device, FLOP/s."""
    v = ctypes.c_double()
    _check(load().perm_measure_fp64_peak(float(ms_target), ctypes.byref(v)), "perm_measure_fp64_peak")
    return v.value


class Plan:
    """A libperm plan: workspace for matrices of order <= n_max of one dtype."""

    def __init__(self, n_max: int, dtype: str = "c128", method: int = METHOD_AUTO, flags: int = 0,
                 mem_budget_bytes: int = 0, max_batch: int = 0, ctas_per_sm: int = 0,
                 low_cols: int = 0):
        lib = load()
        self.dtype = dtype
        self.n_max = n_max
        opts = PermOpts(mem_budget_bytes, max_batch, method, flags, ctas_per_sm, low_cols)
        h = _VP()
        _check(lib.perm_plan_create(int(n_max), DTYPES[dtype], ctypes.byref(opts), ctypes.byref(h)),
               "perm_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        return int(load().perm_plan_workspace_bytes(self._h))

    def describe(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1024)
        load().perm_plan_describe(self._h, buf, 1024)
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().perm_plan_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- device buffers (torch tensors) -------------------------------------------
    def batch(self, mats, sizes: Sequence[int], out, item_status=None, stream=None):
        """Enqueue permanents of concatenated device matrices (torch tensors)."""
        sz = (ctypes.c_int * len(sizes))(*[int(s) for s in sizes])
        rc = load().perm_batch(self._h, _VP(mats.data_ptr() if mats is not None and mats.numel() else 0), sz,
                               len(sizes), _VP(out.data_ptr()),
                               _VP(item_status.data_ptr() if item_status is not None else 0),
                               _VP(_stream_ptr(stream)))
        _check(rc, "perm_batch")

    # -- host buffers (numpy) -------------------------------------------------------
    def batch_host(self, mats: np.ndarray, sizes: Sequence[int], out: np.ndarray,
                   item_status: Optional[np.ndarray] = None, stream=None):
        sz = (ctypes.c_int * len(sizes))(*[int(s) for s in sizes])
        rc = load().perm_batch_host(self._h, _VP(mats.ctypes.data if mats.size else 0), sz, len(sizes),
                                    _VP(out.ctypes.data),
                                    _VP(item_status.ctypes.data if item_status is not None else 0),
                                    _VP(_stream_ptr(stream) if stream is not None else 0))
        _check(rc, "perm_batch_host")


    # -- one matrix split by Ryser code range (device buffers) --------------------------
    def ryser_partials(self, mat, n: int, begin: int, end: int, partials, stream=None):
        """Partial sums of pieces [begin, end) of one order-n device matrix into `partials`."""
        rc = load().perm_ryser_partials(self._h, _VP(mat.data_ptr()), int(n), int(begin), int(end),
                                        _VP(partials.data_ptr()), _VP(_stream_ptr(stream)))
        _check(rc, "perm_ryser_partials")

    def ryser_finish(self, n: int, partials, out, item_status=None, stream=None):
        """The permanent from ALL pieces' partial sums (device, in piece order)."""
        rc = load().perm_ryser_finish(self._h, int(n), _VP(partials.data_ptr()), _VP(out.data_ptr()),
                                      _VP(item_status.data_ptr() if item_status is not None else 0),
                                      _VP(_stream_ptr(stream)))
        _check(rc, "perm_ryser_finish")


def ryser_pieces(n: int, dtype: str):
    """(pieces, bytes per piece) of Ryser's code range for one order-n matrix (host only)."""
    pieces, nbytes = ctypes.c_longlong(), ctypes.c_size_t()
    _check(load().perm_ryser_pieces(int(n), DTYPES[dtype], ctypes.byref(pieces), ctypes.byref(nbytes)),
           "perm_ryser_pieces")
    return int(pieces.value), int(nbytes.value)


def ryser_split(pieces: int, rank: int, world: int):
    """Rank's contiguous share [begin, end) of `pieces` pieces among `world` ranks (host only)."""
    b, e = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().perm_ryser_split(int(pieces), int(rank), int(world), ctypes.byref(b), ctypes.byref(e)),
           "perm_ryser_split")
    return int(b.value), int(e.value)


def colex_subsets(cols: int, rows: int):
    """The rows-subsets of range(cols) in colex order (the order perm_patterns uses)."""
    import itertools
    subs = list(itertools.combinations(range(cols), rows))
    return sorted(subs, key=lambda c: tuple(reversed(c)))


def patterns(mats, stream=None):
    """All collision-free pattern amplitudes of rows x cols complex matrices (host in/out).

    Returns an array (count, C(cols, rows)) ordered like colex_subsets(cols, rows)."""
    import math
    import torch
    mats = np.ascontiguousarray(np.asarray(mats, dtype=np.complex128))
    if mats.ndim == 2:
        mats = mats[None]
    count, rows, cols = mats.shape
    dev = torch.from_numpy(mats.reshape(-1)).cuda()
    out = torch.empty(count * math.comb(cols, rows), dtype=torch.complex128, device="cuda")
    _check(load().perm_patterns(_VP(dev.data_ptr()), count, rows, cols, _VP(out.data_ptr()),
                                _VP(_stream_ptr(stream))), "perm_patterns")
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(count, -1)


def colex_multisets(cols: int, rows: int):
    """Occupation vectors (t_0..t_{cols-1}) of the outputs of perm_patterns_multiset, in order."""
    import itertools
    subs = sorted(itertools.combinations(range(cols + rows - 1), rows), key=lambda c: tuple(reversed(c)))
    out = []
    for sub in subs:
        t = [0] * cols
        for p, x in enumerate(sub):
            t[x - p] += 1
        out.append(tuple(t))
    return out


def patterns_multiset(mats, stream=None):
    """All output-pattern amplitudes (collisions included) of rows x cols complex
    matrices (host in/out): array (count, C(cols+rows-1, rows)) ordered like
    colex_multisets(cols, rows)."""
    import math
    import torch
    mats = np.ascontiguousarray(np.asarray(mats, dtype=np.complex128))
    if mats.ndim == 2:
        mats = mats[None]
    count, rows, cols = mats.shape
    dev = torch.from_numpy(mats.reshape(-1)).cuda()
    out = torch.empty(count * math.comb(cols + rows - 1, rows), dtype=torch.complex128, device="cuda")
    _check(load().perm_patterns_multiset(_VP(dev.data_ptr()), count, rows, cols, _VP(out.data_ptr()),
                                         _VP(_stream_ptr(stream))), "perm_patterns_multiset")
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(count, -1)


def u128_to_int(lo_hi) -> int:
    lo, hi = (int(x) & 0xFFFFFFFFFFFFFFFF for x in lo_hi)
    return lo | (hi << 64)


def words_to_int(words) -> int:
    """Unsigned integer from 64-bit words, least significant first (any count)."""
    v = 0
    for k, w in enumerate(words):
        v |= (int(w) & 0xFFFFFFFFFFFFFFFF) << (64 * k)
    return v


def permanents(mats, dtype: Optional[str] = None, method: int = METHOD_AUTO, flags: int = 0,
               plan: Optional[Plan] = None, return_status: bool = False):
    """Permanents of a list of square numpy matrices (host in, host out).

    Complex input -> numpy complex128 array; integer input -> list of Python ints
    (with FLAG_WIDE in `flags`, or a wide `plan`, exact up to 2^192).
    """
    import torch
    mats = [np.asarray(m) for m in mats]
    if dtype is None:
        if mats and np.iscomplexobj(mats[0]):
            dtype = "c128"
        elif mats and all(np.isin(m, (0, 1)).all() for m in mats):
            dtype = "u01"
        else:
            dtype = "i64"
    sizes = [m.shape[0] for m in mats]
    npdt = np.complex128 if dtype == "c128" else np.int64
    flat = np.concatenate([np.ascontiguousarray(m, dtype=npdt).reshape(-1) for m in mats]) if mats else np.zeros(0, npdt)
    own = plan is None
    if own:
        plan = Plan(max(sizes) if sizes else 0, dtype, method=method, flags=flags)
    try:
        dev = torch.from_numpy(flat).cuda() if flat.size else torch.zeros(0, dtype=torch.complex128 if dtype == "c128" else torch.int64, device="cuda")
        words = 4 if (flags & FLAG_WIDE or (not own and plan.describe().get("out_words") == 4)) else 2
        if dtype == "c128":
            out = torch.empty(len(mats), dtype=torch.complex128, device="cuda")
        else:
            out = torch.empty((len(mats), words), dtype=torch.int64, device="cuda")
        st = torch.empty(len(mats), dtype=torch.int32, device="cuda")
        plan.batch(dev, sizes, out, st)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        s = st.cpu().numpy()
    finally:
        if own:
            plan.close()
    res = o if dtype == "c128" else [words_to_int(r) for r in o]
    return (res, s) if return_status else res


class Server:
    """The continuous-batching server (perm_server_*): submit host matrices, poll results."""

    def __init__(self, mem_budget_bytes: int = 0, max_batch: int = 0, flags: int = 0):
        lib = load()
        opts = PermOpts(mem_budget_bytes, max_batch, METHOD_AUTO, flags, 0, 0)
        h = _VP()
        _check(lib.perm_server_create(ctypes.byref(opts), None, ctypes.byref(h)), "perm_server_create")
        self._h = h
        self._keep = {}

    def try_submit(self, mat, dtype: str):
        """Submit one matrix; returns (True, ticket) or (False, None) when the queue is full."""
        a = np.ascontiguousarray(mat, dtype=np.complex128 if dtype == "c128" else np.int64)
        t = ctypes.c_uint64()
        rc = load().perm_submit(self._h, _VP(a.ctypes.data if a.size else 0), int(a.shape[0]),
                                DTYPES[dtype], ctypes.byref(t))
        if rc == PERM_EAGAIN:
            return False, None
        _check(rc, "perm_submit")
        self._keep[t.value] = dtype
        return True, t.value

    def submit(self, mat, dtype: str) -> int:
        while True:
            ok, t = self.try_submit(mat, dtype)
            if ok:
                return t

    def poll(self, ticket: int):
        """('done', (value, status)), ('pending', None) or ('missing', None)."""
        buf = (ctypes.c_uint64 * 4)()
        st = ctypes.c_int()
        rc = load().perm_poll(self._h, ctypes.c_uint64(ticket), buf, ctypes.byref(st))
        if rc == PERM_EAGAIN:
            return "pending", None
        if rc == PERM_ENOTFOUND:
            return "missing", None
        _check(rc, "perm_poll")
        dtype = self._keep.pop(ticket, "c128")
        if dtype == "c128":
            v = np.frombuffer(bytes(buf), dtype=np.complex128)[0]
        else:
            v = words_to_int(tuple(buf))   # words the server did not write stay zero
        return "done", (v, st.value)

    def wait_all(self, tickets, timeout_s: float = 60.0, sleep_s: float = 0.0002):
        import time as _t
        out = {}
        end = _t.monotonic() + timeout_s
        pending = list(tickets)
        while pending:
            rest = []
            for t in pending:
                state, v = self.poll(t)
                if state == "done":
                    out[t] = v
                elif state == "pending":
                    rest.append(t)
                else:
                    raise LibpermError(PERM_ENOTFOUND, "perm_poll")
            pending = rest
            if pending:
                if _t.monotonic() > end:
                    raise TimeoutError(f"{len(pending)} requests not done")
                _t.sleep(sleep_s)
        return [out[t] for t in tickets]

    def destroy(self, timeout_ms: int = 600000) -> int:
        rc = PERM_OK
        if getattr(self, "_h", None) and self._h.value:
            rc = load().perm_server_destroy(self._h, int(timeout_ms))
            self._h = _VP()
        return rc

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        rc = self.destroy()
        if rc != PERM_OK:
            raise LibpermError(rc, "perm_server_destroy")

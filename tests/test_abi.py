"""The C ABI library loads and exports every function include/libperm.h declares.

CPU-only: no compute call is made; calls that would need a device are only
checked to fail cleanly with a status code."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "libperm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(perm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1802_02779_gb300 import build
    build.build()
    from paper_1802_02779_gb300 import libperm
    return libperm.load()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ("perm_plan_create", "perm_plan_destroy", "perm_batch", "perm_batch_host",
              "perm_server_create", "perm_submit", "perm_poll", "perm_server_destroy",
              "perm_strerror"):
        assert f in fns


def test_every_declared_symbol_is_exported(lib):
    for f in declared_functions():
        assert hasattr(lib, f), f"libperm.so does not export {f}"


def test_binding_covers_the_header():
    from paper_1802_02779_gb300 import libperm
    assert set(declared_functions()) == set(libperm._SIGS)


def test_status_strings(lib):
    from paper_1802_02779_gb300 import libperm
    for code in range(0, 9):
        assert libperm.strerror(code)
    assert libperm.version().count(".") == 2


def test_null_arguments_are_rejected(lib):
    from paper_1802_02779_gb300 import libperm as lp
    assert lib.perm_plan_create(4, lp.PERM_C128, None, None) == lp.PERM_EINVAL
    h = ctypes.c_void_p()
    assert lib.perm_plan_create(-1, lp.PERM_C128, None, ctypes.byref(h)) == lp.PERM_EINVAL
    assert lib.perm_plan_create(41, lp.PERM_C128, None, ctypes.byref(h)) == lp.PERM_EINVAL
    assert lib.perm_plan_create(4, 99, None, ctypes.byref(h)) == lp.PERM_EINVAL
    sizes = (ctypes.c_int * 1)(3)
    assert lib.perm_batch(None, None, sizes, 1, None, None, None) == lp.PERM_EINVAL
    assert lib.perm_plan_destroy(None) == lp.PERM_OK
    assert lib.perm_server_destroy(None, 0) == lp.PERM_OK
    assert lib.perm_submit(None, None, 3, lp.PERM_C128, None) == lp.PERM_EINVAL
    assert lib.perm_poll(None, 1, None, None) == lp.PERM_EINVAL


def test_library_is_built_for_sm103a():
    """The build passes exactly one -gencode for sm_103a."""
    from paper_1802_02779_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def header_constants():
    """Every `PERM_X = v` enumerator and `#define PERM_FLAG_X v` of the header."""
    text = open(HEADER).read()
    consts = {k: int(v) for k, v in re.findall(r"\b(PERM_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    consts.update({k: int(v) for k, v in re.findall(r"#define\s+(PERM_FLAG_[A-Z0-9_]+)\s+(\d+)u", text)})
    return consts


def test_binding_constants_match_the_header():
    from paper_1802_02779_gb300 import libperm as lp
    c = header_constants()
    binding = {
        "PERM_OK": lp.PERM_OK, "PERM_EINVAL": lp.PERM_EINVAL, "PERM_ENOMEM": lp.PERM_ENOMEM,
        "PERM_EOVERFLOW": lp.PERM_EOVERFLOW, "PERM_ECUDA": lp.PERM_ECUDA, "PERM_EAGAIN": lp.PERM_EAGAIN,
        "PERM_ETIMEDOUT": lp.PERM_ETIMEDOUT, "PERM_ESHUTDOWN": lp.PERM_ESHUTDOWN,
        "PERM_ENOTFOUND": lp.PERM_ENOTFOUND,
        "PERM_C128": lp.PERM_C128, "PERM_U01": lp.PERM_U01, "PERM_I64": lp.PERM_I64,
        "PERM_METHOD_AUTO": lp.METHOD_AUTO, "PERM_METHOD_SZ": lp.METHOD_SZ, "PERM_METHOD_RYSER": lp.METHOD_RYSER,
        "PERM_FLAG_PLAIN": lp.FLAG_PLAIN, "PERM_FLAG_GRAPH": lp.FLAG_GRAPH,
        "PERM_FLAG_AUTOTUNE": lp.FLAG_AUTOTUNE, "PERM_FLAG_WIDE": lp.FLAG_WIDE,
    }
    assert set(binding) == set(c)
    for k, v in binding.items():
        assert c[k] == v, k


def test_opts_struct_matches_the_header():
    """perm_opts: the ctypes fields are the header's fields, in order, with the same C types."""
    from paper_1802_02779_gb300 import libperm as lp
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct perm_opts\s*\{(.*?)\}\s*perm_opts;", text, re.S).group(1)
    fields = re.findall(r"(size_t|int|unsigned)\s+([a-z_]+)\s*;", body)
    ctypes_of = {"size_t": ctypes.c_size_t, "int": ctypes.c_int, "unsigned": ctypes.c_uint}
    assert [(n, ctypes_of[t]) for t, n in fields] == list(lp.PermOpts._fields_)

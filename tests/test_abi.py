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

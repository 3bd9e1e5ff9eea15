"""perm_sz_noalloc: the Store-zechin entry point that allocates no device memory.

It is meant for callers that cannot call cudaMalloc (a framework whose pool owns
all device memory, a loop that must not take an allocation's device-wide
synchronisation, a thread that is capturing a CUDA graph).  This test calls it
through the C ABI twice in a row for each matrix and checks every result against
the ordinary entry point, perm_batch with Store-zechin, within the tolerance the
other tests use (1e-12 * per(|A|) for complex input, bit-exact for integers).
It is collected last on purpose and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lp():
    assert torch.cuda.is_available()
    from paper_1802_02779_gb300 import build
    build.build()
    from paper_1802_02779_gb300 import libperm
    libperm.load()
    return libperm


def _noalloc(lp, dev_mat, n, dtype, out, status):
    stream = torch.cuda.current_stream().cuda_stream
    rc = lp.load().perm_sz_noalloc(ctypes.c_void_p(dev_mat.data_ptr() if n else 0), n, lp.DTYPES[dtype],
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                   ctypes.c_void_p(stream))
    return rc


@pytest.mark.parametrize("n", [5, 14, 20, 22])
def test_complex_two_calls_match_perm_batch(lp, n):
    g = np.random.default_rng(4000 + n)
    a = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2 * n)
    dev = torch.from_numpy(a.reshape(-1)).cuda()
    ref = lp.permanents([a], "c128", method=lp.METHOD_SZ)[0]
    tol = 1e-12 * oracle.per_abs(a)
    for _ in range(2):
        out = torch.full((1,), complex("nan+nanj"), dtype=torch.complex128, device="cuda")
        st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        assert _noalloc(lp, dev, n, "c128", out, st) == lp.PERM_OK
        torch.cuda.synchronize()
        got = complex(out.cpu().numpy()[0])
        assert int(st.item()) == lp.PERM_OK
        assert abs(got - ref) <= tol, (n, got, ref)


@pytest.mark.parametrize("n,dtype", [(9, "u01"), (20, "u01"), (23, "u01"), (12, "i64")])
def test_integer_two_calls_match_perm_batch(lp, n, dtype):
    g = np.random.default_rng(5000 + n)
    a = (g.random((n, n)) < 0.6).astype(np.int64) if dtype == "u01" else g.integers(0, 4, size=(n, n)).astype(np.int64)
    dev = torch.from_numpy(a.reshape(-1)).cuda()
    ref = lp.permanents([a], dtype, method=lp.METHOD_SZ)[0]
    for _ in range(2):
        out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        st = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        assert _noalloc(lp, dev, n, dtype, out, st) == lp.PERM_OK
        torch.cuda.synchronize()
        assert int(st.item()) == lp.PERM_OK
        assert lp.u128_to_int(out.cpu().numpy()) == ref


def test_limits_and_empty(lp):
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    big = torch.zeros(24 * 24, dtype=torch.int64, device="cuda")
    assert _noalloc(lp, big, 24, "u01", out, st) == lp.PERM_EINVAL
    bigc = torch.zeros(23 * 23, dtype=torch.complex128, device="cuda")
    outc = torch.zeros(1, dtype=torch.complex128, device="cuda")
    assert _noalloc(lp, bigc, 23, "c128", outc, st) == lp.PERM_EINVAL
    assert _noalloc(lp, big, 0, "u01", out, st) == lp.PERM_OK
    torch.cuda.synchronize()
    assert lp.u128_to_int(out.cpu().numpy()) == 1

"""perm_sz_noalloc: the Store-zechin entry point that allocates no device memory.

It is meant for callers that cannot call cudaMalloc: code inside a framework
whose memory pool owns all device memory, and loops that must not take an
allocation's device-wide synchronisation.  Its chain tables live in a fixed
64 MiB scratch array in the library's device image, so it accepts complex
orders up to 22 and integer orders up to 23.

This test calls it through the C ABI twice in a row for each matrix and checks:
  * every result is bit-identical to the ordinary entry point, perm_batch with
    Store-zechin (the header's promise; both sum every table entry over its
    columns in ascending order), which is within any tolerance the other tests
    use;
  * every result against the oracle (1e-12 * per(|A|) for complex input,
    bit-exact for integers);
  * the device's free memory is the same before and after a call (after the
    first call on the device has done its one-time set-up).
It is collected last on purpose and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tests.gpu_helpers import oracle_c, oracle_i

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


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("n", [5, 14, 20, 22])
def test_complex_two_calls_match_perm_batch(lp, n):
    g = np.random.default_rng(4000 + n)
    a = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2 * n)
    dev = torch.from_numpy(a.reshape(-1)).cuda()
    ref = lp.permanents([a], "c128", method=lp.METHOD_SZ)[0]
    want = oracle_c(a)
    tol = 1e-12 * oracle.per_abs(a)
    outs = [torch.full((1,), complex("nan+nanj"), dtype=torch.complex128, device="cuda") for _ in range(2)]
    sts = [torch.full((1,), -7, dtype=torch.int32, device="cuda") for _ in range(2)]
    assert _noalloc(lp, dev, n, "c128", outs[0], sts[0]) == lp.PERM_OK   # set-up on first use
    free0 = _free_bytes()
    assert _noalloc(lp, dev, n, "c128", outs[1], sts[1]) == lp.PERM_OK
    assert _free_bytes() == free0
    for out, st in zip(outs, sts):
        got = complex(out.cpu().numpy()[0])
        assert int(st.item()) == lp.PERM_OK
        assert got == ref, (n, got, ref)                     # bit-identical to perm_batch
        assert abs(got - want) <= tol, (n, got, want)        # and within the oracle's tolerance


@pytest.mark.parametrize("n,dtype", [(9, "u01"), (20, "u01"), (23, "u01"), (12, "i64")])
def test_integer_two_calls_match_perm_batch(lp, n, dtype):
    g = np.random.default_rng(5000 + n)
    a = (g.random((n, n)) < 0.6).astype(np.int64) if dtype == "u01" else g.integers(0, 4, size=(n, n)).astype(np.int64)
    dev = torch.from_numpy(a.reshape(-1)).cuda()
    ref = lp.permanents([a], dtype, method=lp.METHOD_SZ)[0]
    want = oracle_i(a)
    assert ref == want
    outs = [torch.full((2,), -1, dtype=torch.int64, device="cuda") for _ in range(2)]
    sts = [torch.full((1,), -7, dtype=torch.int32, device="cuda") for _ in range(2)]
    assert _noalloc(lp, dev, n, dtype, outs[0], sts[0]) == lp.PERM_OK
    free0 = _free_bytes()
    assert _noalloc(lp, dev, n, dtype, outs[1], sts[1]) == lp.PERM_OK
    assert _free_bytes() == free0
    for out, st in zip(outs, sts):
        assert int(st.item()) == lp.PERM_OK
        assert lp.u128_to_int(out.cpu().numpy()) == want


def test_limits_and_empty(lp):
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    big = torch.zeros(24 * 24, dtype=torch.int64, device="cuda")
    assert _noalloc(lp, big, 24, "u01", out, st) == lp.PERM_EINVAL
    bigc = torch.zeros(23 * 23, dtype=torch.complex128, device="cuda")
    outc = torch.zeros(1, dtype=torch.complex128, device="cuda")
    assert _noalloc(lp, bigc, 23, "c128", outc, st) == lp.PERM_EINVAL
    assert _noalloc(lp, big, -1, "u01", out, st) == lp.PERM_EINVAL
    assert _noalloc(lp, big, 0, "u01", out, st) == lp.PERM_OK
    torch.cuda.synchronize()
    assert lp.u128_to_int(out.cpu().numpy()) == 1

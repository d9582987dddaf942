"""The allocation-free Gram entry point, for callers that must not allocate
device memory (a fixed device-memory budget held by another allocator, or a
loop that cannot take cudaFree's implicit synchronisation).

It is checked through the C ABI against the allocating bbl_block_gram on two
calls in a row (the shared scratch array keeps the first call's contents),
with the tolerance the kernel tests use for a reordered FP64 sum, and a
request beyond its fixed scratch must be refused with a clear error.  This
file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53


def _noalloc(lib, basis, W, Cout, dtype_code, torch):
    nb, n, b = basis.shape
    return lib.bbl_block_gram_noalloc(n, b, nb, dtype_code, C.c_void_p(basis.data_ptr()), C.c_void_p(W.data_ptr()),
                                      C.c_void_p(Cout.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _allocating(lib, basis, W, Cout, dtype_code, torch):
    nb, n, b = basis.shape
    return lib.bbl_block_gram(n, b, nb, dtype_code, C.c_void_p(basis.data_ptr()), C.c_void_p(W.data_ptr()),
                              C.c_void_p(Cout.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_noalloc_gram_matches_allocating_gram_on_two_calls(dtype):
    torch, bbl = need_gpu()
    from paper_2210_15763_gb300 import _lib
    lib = _lib.load()
    code = _lib.FP64 if dtype == "fp64" else _lib.FP32
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    # two different problems in a row: sizes, blocks and values change between the calls
    for (n, b, nb, seed) in ((50_001, 8, 13, 1), (8_191, 4, 40, 2)):
        rng = np.random.default_rng(seed)
        Q = to_dev(torch, rng.standard_normal((nb, n, b)), tdt)
        W = to_dev(torch, rng.standard_normal((n, b)), tdt)
        got = torch.empty((nb * b, b), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(got)
        assert _noalloc(lib, Q, W, got, code, torch) == 0, lib.bbl_last_error()
        assert _allocating(lib, Q, W, ref, code, torch) == 0, lib.bbl_last_error()
        Qh = Q.double().cpu().numpy()
        Wh = W.double().cpu().numpy()
        bound = np.concatenate([np.abs(Qh[j]).T @ np.abs(Wh) for j in range(nb)])
        tol = (64 * EPS64 if dtype == "fp64" else 64 * 2.0 ** -24) * bound
        assert np.all(np.abs(got.cpu().numpy() - ref.cpu().numpy()) <= tol)


def test_noalloc_gram_rejects_requests_beyond_its_scratch():
    torch, bbl = need_gpu()
    from paper_2210_15763_gb300 import _lib
    lib = _lib.load()
    n, b, nb = 1000, 16, 4200        # nb*b*b = 1,075,200 > 2^20 partial sums
    Q = torch.zeros((nb, n, b), dtype=torch.float32, device="cuda")
    W = torch.zeros((n, b), dtype=torch.float32, device="cuda")
    out = torch.empty((nb * b, b), dtype=torch.float64, device="cuda")
    st = _noalloc(lib, Q, W, out, _lib.FP32, torch)
    assert _lib.STATUS[st] == "BBL_ERR_INVALID_ARG"
    assert b"exceeds the fixed scratch" in lib.bbl_last_error()

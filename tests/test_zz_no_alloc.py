"""The allocation-free Gram entry point, for callers that must not allocate
device memory (a fixed device-memory budget held by another allocator, or a
loop that cannot take cudaFree's implicit synchronisation).

It is checked through the C ABI on calls in a row (the shared scratch array
keeps the last call's contents) against the FP64 host product Q^T W, within
the bound the kernel tests use for a reordered sum, and against the
allocating bbl_block_gram.  The cases cover one column group, many column
groups (more chunk tickets than a 64-double ticket area would hold), and a
worker count limited by the scratch capacity; a request beyond the fixed
scratch must be refused with a clear error.  This file is collected last so
that a run stopping at its first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24
SCRATCH_PARTIALS = 2 ** 20 - 2048     # partial sums the fixed array holds


def _noalloc(lib, basis, W, Cout, dtype_code, torch):
    nb, n, b = basis.shape
    return lib.bbl_block_gram_noalloc(n, b, nb, dtype_code, C.c_void_p(basis.data_ptr()), C.c_void_p(W.data_ptr()),
                                      C.c_void_p(Cout.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _allocating(lib, basis, W, Cout, dtype_code, torch):
    nb, n, b = basis.shape
    return lib.bbl_block_gram(n, b, nb, dtype_code, C.c_void_p(basis.data_ptr()), C.c_void_p(W.data_ptr()),
                              C.c_void_p(Cout.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _check_sequence(cases, dtype):
    torch, bbl = need_gpu()
    from paper_2210_15763_gb300 import _lib
    lib = _lib.load()
    code = _lib.FP64 if dtype == "fp64" else _lib.FP32
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    eps = EPS64 if dtype == "fp64" else EPS32
    for (n, b, nb, seed) in cases:
        assert nb * b * b <= SCRATCH_PARTIALS
        rng = np.random.default_rng(seed)
        Q = to_dev(torch, rng.standard_normal((nb, n, b)), tdt)
        W = to_dev(torch, rng.standard_normal((n, b)), tdt)
        got = torch.empty((nb * b, b), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(got)
        assert _noalloc(lib, Q, W, got, code, torch) == 0, lib.bbl_last_error()
        assert _allocating(lib, Q, W, ref, code, torch) == 0, lib.bbl_last_error()
        Qh = Q.double().cpu().numpy().transpose(0, 2, 1).reshape(nb * b, n)   # rows = basis columns
        Wh = W.double().cpu().numpy()
        exact = Qh @ Wh
        bound = np.abs(Qh) @ np.abs(Wh)
        tol = 64 * eps * bound
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.abs(g - exact) <= tol), (n, b, nb, float(np.max(np.abs(g - exact) / np.maximum(bound, 1e-300))))
        assert np.all(np.abs(g - r) <= 2 * tol), (n, b, nb)


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_noalloc_gram_matches_host_product_and_allocating_gram_on_two_calls(dtype):
    # two different problems in a row: sizes, blocks and values change between the calls
    _check_sequence(((50_001, 8, 13, 1), (8_191, 4, 40, 2)), dtype)


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_noalloc_gram_many_column_groups_and_capacity_limited_workers(dtype):
    # b = 1 with 40,000 blocks: 157 column groups, each with its own chunk
    # ticket; b = 16 with 4,080 blocks: 1,044,480 partial sums, so the fixed
    # array holds one worker's partials only (every column group walks all
    # row chunks alone); then a small case again, after the large ones
    _check_sequence(((700, 1, 40_000, 3), (64, 16, 4_080, 4), (3_001, 8, 5, 5)), dtype)


def test_noalloc_gram_rejects_requests_beyond_its_scratch():
    torch, bbl = need_gpu()
    from paper_2210_15763_gb300 import _lib
    lib = _lib.load()
    n, b, nb = 1000, 16, 4200        # nb*b*b = 1,075,200 > 2^20 - 2048 partial sums
    Q = torch.zeros((nb, n, b), dtype=torch.float32, device="cuda")
    W = torch.zeros((n, b), dtype=torch.float32, device="cuda")
    out = torch.empty((nb * b, b), dtype=torch.float64, device="cuda")
    st = _noalloc(lib, Q, W, out, _lib.FP32, torch)
    assert _lib.STATUS[st] == "BBL_ERR_INVALID_ARG"
    assert b"exceeds the fixed scratch" in lib.bbl_last_error()

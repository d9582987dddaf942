"""The tiled stored format (BBL_TILED) against the oracle's SpMM.

The tiled SpMM sums each output row's products in a different order than
the oracle (tile by tile, rows of a tile from shared memory), so the two
differ by rounding only: |W_gpu - W_ref| <= 64 * eps * (|H| |V|) entrywise,
eps of the arithmetic (FP64, FP32).  Block sizes below 16 bytes of elements
fall back to the CSR copy and must give the same result.
"""
import numpy as np
import pytest

import synth
from oracle.spmm import spmm as ospmm, spmm_rows
from tests.gpu_util import abs_bound, need_gpu, to_dev

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def _mat(kind):
    if kind == "ragged":
        return synth.random_sparse_symmetric(1037, 7, seed=11, empty_rows=5, long_row=300)
    if kind == "kron":
        return synth.kron_matrix("kron_n2e4", scale=0.4)     # 80 x 40 factors
    if kind == "lap2d":
        return synth.laplacian_2d(33, 31)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["ragged", "kron", "lap2d"])
@pytest.mark.parametrize("tile", [16, 40, 100, 1024])
@pytest.mark.parametrize("b", [1, 2, 4, 8, 16])
def test_tiled_spmm_fp64_and_fp32(kind, tile, b):
    torch, bbl = need_gpu()
    A = _mat(kind)
    V = np.random.default_rng(b + tile).standard_normal((A.n, b))
    ref = ospmm(A, V)
    M = bbl.Matrix(A, storage="fp64", fmt="tiled", sell_sigma=tile)
    W = bbl.spmm(M, to_dev(torch, V)).cpu().numpy()
    assert np.all(np.abs(W - ref) <= 64 * EPS64 * abs_bound(A, V) + 1e-300)
    A32 = synth.CSR(A.n, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    V32 = V.astype(np.float32).astype(np.float64)
    M32 = bbl.Matrix(A32, storage="fp32", fmt="tiled", sell_sigma=tile)
    W32 = bbl.spmm(M32, to_dev(torch, V32, torch.float32)).cpu().numpy().astype(np.float64)
    ref32 = ospmm(A32, V32)
    bound = abs_bound(A32, V32)
    assert np.all(np.abs(W32 - ref32) <= 64 * EPS32 * bound + 1e-30)
    # FP64 arithmetic on the FP32 values (the residual product of the mixed form)
    W64 = bbl.spmm_f64(M32, to_dev(torch, V32)).cpu().numpy()
    assert np.all(np.abs(W64 - ref32) <= 64 * EPS64 * bound + 1e-300)


def test_tiled_mixed_precision_solve_matches_oracle():
    """FP32 stage and float-float polish on the tiled format (the polish's
    SpMM runs float-float blocks through the tiled kernel)."""
    from oracle import lanczos as OL
    from oracle import rng as OR
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    piv = OR.normal_block(7, H.n, 8)
    ref = OL.block_lanczos(H, 8, 8, piv, tol=1e-9)
    M = bbl.Matrix(H, storage="fp32", fmt="tiled", sell_sigma=100)
    res = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9)
    assert res.converged and res.stats["polish_iters"] >= 1
    np.testing.assert_allclose(res.evals, ref.evals, rtol=1e-10)


def test_tiled_rejects_a_tile_pair_beyond_16_bit_offsets():
    torch, bbl = need_gpu()
    n = 300
    d = np.random.default_rng(1).standard_normal((n, n))
    A = synth.csr_from_dense(d + d.T)        # 90,000 entries in one (row block, column tile) pair
    with pytest.raises(bbl.BBLError) as e:
        bbl.Matrix(A, storage="fp32", fmt="tiled", sell_sigma=n)
    assert e.value.status == 8
    M = bbl.Matrix(A, storage="fp32", fmt="tiled", sell_sigma=128)   # 16,384 per pair at most
    V = np.random.default_rng(2).standard_normal((n, 8)).astype(np.float32)
    W = bbl.spmm(M, to_dev(torch, V)).cpu().numpy()
    ref = ospmm(A, V.astype(np.float64))
    assert np.all(np.abs(W - ref) <= 64 * EPS32 * abs_bound(A, V.astype(np.float64)))


def test_tiled_fullsize_spmm_sampled_rows():
    """n = 2,000,000 (kron_n2e6, 564.8 M nonzeros) in the benchmark's tiled
    configuration (tile 1000, FP32, b = 8) against the oracle's rows."""
    torch, bbl = need_gpu()
    A = synth.kron_matrix("kron_n2e6", fp32_values=True)
    M = bbl.Matrix(A, storage="fp32", fmt="tiled", sell_sigma=1000)
    V = np.random.default_rng(3).standard_normal((A.n, 8)).astype(np.float32)
    W = bbl.spmm(M, to_dev(torch, V)).cpu().numpy().astype(np.float64)
    rows = np.unique(np.concatenate([np.sort(np.random.default_rng(4).choice(A.n, 2000, replace=False)),
                                     [0, 999, 1000, A.n - 1]]))
    V64 = V.astype(np.float64)
    ref = spmm_rows(A, V64, rows)
    Habs = synth.CSR(A.n, A.row_ptr, A.col, np.abs(A.val.astype(np.float64)))
    bound = 64 * EPS32 * spmm_rows(Habs, np.abs(V64), rows)
    assert np.all(np.abs(W[rows] - ref) <= bound)

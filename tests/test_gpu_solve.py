"""Whole-solver parity of bbl_solve with the oracle, plus method behaviour.

FP64 tolerance: the nev eigenvalues agree with the oracle's to relative 1e-10
(both are Ritz values of the same Krylov space, converged to residual
1e-8*||H||_inf; the Ritz values are then accurate to about
resid^2/gap, far below 1e-10).  Mixed precision with the FP64 polish must
meet the same bar; the FP32 stage alone must be within relative 1e-6.
"""
import numpy as np
import pytest

import synth
from oracle import lanczos as OL
from oracle import pivot as OP
from oracle import rng as OR
from oracle.spmm import norm_inf, spmm as ospmm
from tests.gpu_util import need_gpu, principal_angle_sin, to_dev

pytestmark = pytest.mark.gpu


def _check_eigs(res, ref_evals, H, tol, rel=1e-10):
    np.testing.assert_allclose(res.evals, ref_evals, rtol=rel, atol=rel * 1e-3)
    X = res.evecs.cpu().numpy() if hasattr(res.evecs, "cpu") else res.evecs
    assert np.abs(X.T @ X - np.eye(X.shape[1])).max() < 1e-8
    R = ospmm(H, X) - X * res.evals
    true_res = np.linalg.norm(R, axis=0)
    assert np.all(true_res <= tol * norm_inf(H) * 1.01)
    np.testing.assert_allclose(res.resid, true_res, rtol=1e-6, atol=1e-14 * norm_inf(H))
    return X


@pytest.mark.parametrize("b", [1, 2, 4, 8, 16])
def test_solve_fp64_kron_small_vs_oracle(b):
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.3)  # n = 60 x 30
    nev = 4
    piv = OR.normal_block(5, H.n, b)
    ref = OL.block_lanczos(H, nev, b, piv, tol=1e-8)
    M = bbl.Matrix(H)
    res = bbl.solve(M, nev, b, pivot=piv, tol=1e-8, check_every=1)
    assert res.converged and ref.converged
    _check_eigs(res, ref.evals, H, 1e-8)
    assert abs(res.stats["iters"] - ref.iters) <= 1
    # eigenvectors: same sign convention, same vectors (the spectrum is simple here)
    X = res.evecs.cpu().numpy()
    assert np.abs(X - ref.evecs).max() < 1e-6


def test_solve_fp64_full_size_config_n2e4_vs_oracle():
    """The plain FP64 configuration: n = 20,000, ~100 nnz/row, b = 4, nev = 4."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4")
    piv = OR.normal_block(20221028, H.n, 4)
    ref = OL.block_lanczos(H, 4, 4, piv, tol=1e-8)
    res = bbl.solve(bbl.Matrix(H), 4, 4, pivot=piv, tol=1e-8, check_every=1)
    assert res.converged
    _check_eigs(res, ref.evals, H, 1e-8)
    assert abs(res.stats["iters"] - ref.iters) <= 1
    assert res.stats["ritz_solves"] >= res.stats["iters"]


def test_adaptive_convergence_tests_stop_within_a_few_blocks_of_the_oracle():
    """check_every=0 (the default) tests convergence at predicted blocks only:
    far fewer Ritz solves, the same eigenpairs, and a stop at most a few
    blocks after the first block that passes (the oracle tests every block)."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4")
    piv = OR.normal_block(20221028, H.n, 4)
    ref = OL.block_lanczos(H, 4, 4, piv, tol=1e-8)
    res = bbl.solve(bbl.Matrix(H), 4, 4, pivot=piv, tol=1e-8)
    assert res.converged
    _check_eigs(res, ref.evals, H, 1e-8)
    assert ref.iters - 1 <= res.stats["iters"] <= ref.iters + 4
    assert res.stats["ritz_solves"] < 0.6 * res.stats["iters"]


def test_solve_random_pivot_null_uses_the_published_generator():
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.3)
    ref = OL.block_lanczos(H, 4, 4, OP.random_pivot(H.n, 4, 99), tol=1e-8)
    res = bbl.solve(bbl.Matrix(H), 4, 4, pivot=None, seed=99, tol=1e-8, check_every=1)
    _check_eigs(res, ref.evals, H, 1e-8)
    assert abs(res.stats["iters"] - ref.iters) <= 1


def test_ritz_solve_in_line_matches_the_side_stream():
    """ritz_overlap = 0 runs each Ritz solve on the caller's stream before the
    next block, 2 on the side stream with the next Gram-Schmidt waiting for
    it; all report the same block, eigenvalues and vectors as the default;
    other values are refused."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    piv = OR.normal_block(12, H.n, 4)
    M = bbl.Matrix(H)
    r1 = bbl.solve(M, 4, 4, pivot=piv, tol=1e-9, check_every=1, ritz_overlap=1)
    for mode in (0, 2):
        r0 = bbl.solve(M, 4, 4, pivot=piv, tol=1e-9, check_every=1, ritz_overlap=mode)
        assert r0.converged and r1.converged
        assert r0.stats["iters"] == r1.stats["iters"]
        np.testing.assert_allclose(r0.evals, r1.evals, rtol=1e-13)
        X0, X1 = r0.evecs.cpu().numpy(), r1.evecs.cpu().numpy()
        assert np.abs(X0 - X1).max() < 1e-10
    with pytest.raises(RuntimeError, match="ritz_overlap"):
        bbl.solve(M, 4, 4, pivot=piv, tol=1e-9, ritz_overlap=3)


def test_solve_laplacian_1d_closed_form_b1():
    torch, bbl = need_gpu()
    n = 300
    H = synth.laplacian_1d(n)
    k = np.arange(1, n + 1)
    want = np.sort(2 - 2 * np.cos(k * np.pi / (n + 1)))[:3]
    res = bbl.solve(bbl.Matrix(H), 3, 1, pivot=OR.normal_block(1, n, 1), tol=1e-10, max_vectors=n)
    assert res.converged
    np.testing.assert_allclose(res.evals, want, rtol=1e-10)


def test_solve_laplacian_2d_multiplicities():
    torch, bbl = need_gpu()
    nx = 24
    H = synth.laplacian_2d(nx, nx)
    e1 = np.sort(2 - 2 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1)))
    want = np.sort((e1[:, None] + e1[None, :]).ravel())[:6]
    res = bbl.solve(bbl.Matrix(H), 6, 4, pivot=OR.normal_block(2, H.n, 4), tol=1e-10)
    assert res.converged
    np.testing.assert_allclose(res.evals, want, rtol=1e-10)


def test_solve_exact_pivot_converges_in_one_block():
    torch, bbl = need_gpu()
    A = synth.random_sparse_symmetric(300, 6, seed=33)
    w, U = np.linalg.eigh(A.to_dense())
    res = bbl.solve(bbl.Matrix(A), 4, 4, pivot=U[:, :4].copy(), tol=1e-10)
    assert res.converged and res.stats["iters"] == 1
    np.testing.assert_allclose(res.evals, w[:4], rtol=1e-12)


def test_solve_symmetry_sector_pivot_misses_the_odd_ground_state():
    import scipy.sparse as sp
    torch, bbl = need_gpu()
    n = 120
    A = synth.random_sparse_symmetric(n, 6, seed=5).to_scipy()
    J = sp.csr_matrix((np.ones(n), (np.arange(n), np.arange(n)[::-1])), shape=(n, n))
    H = synth.csr_from_scipy(A + J @ A @ J)
    w, U = np.linalg.eigh(H.to_dense())
    parity = np.sign(np.sum(U * U[::-1], axis=0))
    p = OR.normal_block(3, n, 2)
    even = 0.5 * (p + p[::-1])
    res = bbl.solve(bbl.Matrix(H), 3, 2, pivot=even, tol=1e-9, max_vectors=60)
    np.testing.assert_allclose(res.evals, w[parity > 0][:3], rtol=1e-9)


@pytest.mark.parametrize("fmt", ["csr", "sell"])
def test_solve_mixed_precision_with_polish_matches_fp64_oracle(fmt):
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    piv = OR.normal_block(7, H.n, 8)
    ref = OL.block_lanczos(H, 8, 8, piv, tol=1e-8)
    M = bbl.Matrix(H, storage="fp32", fmt=fmt, sell_sigma=256)
    res = bbl.solve(M, 8, 8, pivot=piv, tol=1e-8)
    assert res.converged
    _check_eigs(res, ref.evals, H, 1e-8)
    assert res.stats["polish_iters"] >= 1


@pytest.mark.parametrize("fmt", ["csr", "sell"])
def test_float_float_polish_agrees_with_fp64_polish(fmt):
    """polish=1 keeps the restart's blocks as float-float pairs (~48 bits);
    polish=2 runs it in FP64.  Both reach the FP64 residual bar, give the
    oracle's eigenvalues to 1e-10 and take nearly the same number of blocks."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    piv = OR.normal_block(9, H.n, 8)
    ref = OL.block_lanczos(H, 8, 8, piv, tol=1e-9)
    M = bbl.Matrix(H, storage="fp32", fmt=fmt, sell_sigma=256, keep_fp64=True)
    r1 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, polish=1, check_every=1)
    r2 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, polish=2, check_every=1)
    assert r1.converged and r2.converged
    _check_eigs(r1, ref.evals, H, 1e-9)
    _check_eigs(r2, ref.evals, H, 1e-9)
    np.testing.assert_allclose(r1.evals, r2.evals, rtol=1e-12)
    assert r1.stats["iters"] == r2.stats["iters"]
    assert abs(r1.stats["polish_iters"] - r2.stats["polish_iters"]) <= 1


@pytest.mark.parametrize("nev", [8, 16])
def test_solve_mixed_precision_b16_matches_fp64_oracle(nev):
    """Block size 16 in the mixed-precision form (FP32 stage + float-float
    polish) against the oracle's block Lanczos at b = 16."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    piv = OR.normal_block(17, H.n, 16)
    ref = OL.block_lanczos(H, nev, 16, piv, tol=1e-8)
    M = bbl.Matrix(H, storage="fp32", fmt="sell", sell_sigma=256)
    res = bbl.solve(M, nev, 16, pivot=piv, tol=1e-8)
    assert res.converged
    _check_eigs(res, ref.evals, H, 1e-8)


def test_solve_mixed_precision_stage1_error_below_1e6():
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    piv = OR.normal_block(7, H.n, 8)
    ref = OL.block_lanczos(H, 8, 8, piv, tol=1e-8)
    M = bbl.Matrix(H, storage="fp32", fmt="sell", sell_sigma=256)
    res = bbl.solve(M, 8, 8, pivot=piv, tol=2e-6, polish=0)
    rel = np.abs(res.evals - ref.evals) / np.abs(ref.evals)
    assert rel.max() <= 1e-6, rel


def test_bootstrap_pivot_matches_oracle_subspace():
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.4)
    trunc = 600
    Po, S, th = OP.bootstrap_pivot(H, trunc, 4)
    M = bbl.Matrix(H)
    Pg = bbl.pivot_bootstrap(M, trunc, 4, sub_tol=1e-11).cpu().numpy()
    # same support, same (orthonormal) subspace
    assert set(np.nonzero(np.abs(Pg).sum(axis=1))[0]) <= set(S.tolist())
    Qg, _ = np.linalg.qr(Pg)
    assert principal_angle_sin(Qg, Po) < 1e-6


def test_bootstrap_fp32_sub_solve_gives_an_equally_good_pivot():
    """From an FP32-stored matrix a sub-solve to sub_tol >= 1e-5 runs in FP32:
    its pivot lies in the same truncated space, its Rayleigh-Ritz values on
    H match the FP64 sub-solve's to the sub-solve tolerance, and the main
    solve from it takes the same number of blocks (+-2)."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.6, fp32_values=True)
    trunc = 1500
    M32 = bbl.Matrix(H, storage="fp32")
    M64 = bbl.Matrix(H)
    S = set(OP.truncated_set(H.diagonal(), trunc).tolist())
    P32 = bbl.pivot_bootstrap(M32, trunc, 8, sub_tol=1e-4)
    P64 = bbl.pivot_bootstrap(M64, trunc, 8, sub_tol=1e-4)
    assert set(np.nonzero(np.abs(P32.cpu().numpy()).sum(axis=1))[0]) <= S
    th32, _ = bbl.pivot_rr_residual(M64, P32)
    th64, _ = bbl.pivot_rr_residual(M64, P64)
    nrm = np.abs(H.to_scipy()).sum(axis=1).max()
    np.testing.assert_allclose(th32, th64, rtol=0, atol=1e-4 * nrm)
    r32 = bbl.solve(M32, 8, 8, pivot=P32, tol=1e-8, max_vectors=1200, check_every=1)
    r64 = bbl.solve(M32, 8, 8, pivot=P64, tol=1e-8, max_vectors=1200, check_every=1)
    assert r32.converged and r64.converged
    assert abs(r32.stats["iters"] - r64.stats["iters"]) <= 2
    np.testing.assert_allclose(r32.evals, r64.evals, rtol=1e-11)


def test_bootstrap_pivot_full_space_gives_one_block():
    torch, bbl = need_gpu()
    A = synth.random_sparse_symmetric(200, 6, seed=8)
    M = bbl.Matrix(A)
    P = bbl.pivot_bootstrap(M, A.n, 4, sub_tol=1e-12)
    res = bbl.solve(M, 4, 4, pivot=P, tol=1e-9)
    assert res.converged and res.stats["iters"] == 1


def test_bootstrap_small_truncation_pads_random_columns():
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.2)
    M = bbl.Matrix(H)
    P = bbl.pivot_bootstrap(M, 2, 4, seed=5).cpu().numpy()
    S = OP.truncated_set(H.diagonal(), 2)
    assert np.count_nonzero(P[:, 0]) == 1 and np.count_nonzero(P[:, 1]) == 1
    assert set(np.nonzero(P[:, :2])[0]) == set(S.tolist())
    # Box-Muller through two math libraries: equal to a few ulps
    np.testing.assert_allclose(P[:, 2:], OR.normal_block(5, H.n, 4)[:, 2:], rtol=1e-12, atol=1e-14)


def test_pivot_overlap_matches_oracle_and_flags_the_missing_sector():
    """bbl_pivot_overlap against the oracle's Householder-QR overlap (host and
    device inputs, a rank-deficient pivot), then the diagnostic on the
    symmetry-sector case: the even pivot's overlap with the true odd-sector
    eigenvectors is zero, and the eigenvectors the solve converges to from
    that pivot all overlap it."""
    import scipy.sparse as sp
    torch, bbl = need_gpu()
    rng = np.random.default_rng(12)
    n = 5000
    P = rng.standard_normal((n, 4))
    P[:, 3] = P[:, 0] - 2.0 * P[:, 1]
    X, _ = np.linalg.qr(rng.standard_normal((n, 8)))
    X[:, 0] = np.linalg.qr(P[:, :1])[0][:, 0]
    want = OP.pivot_overlap(P, X)
    np.testing.assert_allclose(bbl.pivot_overlap(P, X), want, atol=1e-12)
    np.testing.assert_allclose(bbl.pivot_overlap(to_dev(torch, P), to_dev(torch, X)), want, atol=1e-12)
    assert abs(want[0] - 1.0) < 1e-12
    n = 120
    A = synth.random_sparse_symmetric(n, 6, seed=5).to_scipy()
    J = sp.csr_matrix((np.ones(n), (np.arange(n), np.arange(n)[::-1])), shape=(n, n))
    H = synth.csr_from_scipy(A + J @ A @ J)
    w, U = np.linalg.eigh(H.to_dense())
    parity = np.sign(np.sum(U * U[::-1], axis=0))
    p = OR.normal_block(3, n, 2)
    even = 0.5 * (p + p[::-1])
    o_true = bbl.pivot_overlap(even, U[:, :6].copy())
    assert np.all(o_true[parity[:6] < 0] < 1e-12) and np.all(o_true[parity[:6] > 0] > 1e-3)
    res = bbl.solve(bbl.Matrix(H), 3, 2, pivot=even, tol=1e-9, max_vectors=60)
    assert np.all(bbl.pivot_overlap(even, res.evecs) > 1e-3)


# ----------------------------------------------------------------- errors
def test_invalid_csr_is_rejected_before_solving():
    torch, bbl = need_gpu()
    A = synth.random_sparse_symmetric(50, 4, seed=1)
    bad = synth.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    bad.col[3] = 10_000
    with pytest.raises(bbl.BBLError) as e:
        bbl.Matrix(bad)
    assert e.value.status == 1
    uns = synth.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    r = int(np.argmax(np.diff(A.row_ptr)))
    s0 = A.row_ptr[r]
    uns.col[s0], uns.col[s0 + 1] = uns.col[s0 + 1], uns.col[s0]
    with pytest.raises(bbl.BBLError):
        bbl.Matrix(uns)


def test_asymmetric_matrix_is_detected_when_asked():
    torch, bbl = need_gpu()
    A = synth.random_sparse_symmetric(50, 4, seed=1)
    asym = synth.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    k = int(np.nonzero(A.col != np.repeat(np.arange(A.n), np.diff(A.row_ptr)))[0][0])
    asym.val[k] += 1.0
    bbl.Matrix(asym)  # accepted without the check
    with pytest.raises(bbl.BBLError) as e:
        bbl.Matrix(asym, check_symmetry=True)
    assert e.value.status == 2


def test_bad_arguments_and_not_converged():
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.3)
    M = bbl.Matrix(H)
    with pytest.raises(bbl.BBLError):
        bbl.solve(M, 4, 17)
    with pytest.raises(bbl.BBLError):
        bbl.solve(M, 0, 4)
    res = bbl.solve(M, 4, 4, pivot=OR.normal_block(5, H.n, 4), tol=1e-12, max_vectors=12)
    assert res.status == "BBL_ERR_NOT_CONVERGED" and res.stats["iters"] == 3
    assert np.all(np.isfinite(res.evals)) and np.all(res.resid > 0)


def test_workspace_cache_reuses_the_bases_across_calls_and_streams():
    """The bases stay cached after a call and the next call of the same size
    takes them (no growth); a call on another stream shares them (its reuse
    is ordered by an event); release empties the cache.  Results agree to
    rounding (the persistent Gram kernels sum their chunks in ticket order)."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    M = bbl.Matrix(H, storage="fp32")
    bbl.workspace_release()
    assert bbl.workspace_bytes() == 0
    r1 = bbl.solve(M, 4, 4, pivot=None, seed=3, tol=1e-8, max_vectors=400)
    held = bbl.workspace_bytes()
    assert held > 0
    r2 = bbl.solve(M, 4, 4, pivot=None, seed=3, tol=1e-8, max_vectors=400)
    assert bbl.workspace_bytes() == held
    side = torch.cuda.Stream()
    r3 = bbl.solve(M, 4, 4, pivot=None, seed=3, tol=1e-8, max_vectors=400, stream=side)
    torch.cuda.synchronize()
    assert bbl.workspace_bytes() == held
    for r in (r1, r2, r3):
        assert r.converged
    np.testing.assert_allclose(r2.evals, r1.evals, rtol=1e-12)
    np.testing.assert_allclose(r3.evals, r1.evals, rtol=1e-12)
    bbl.workspace_release()
    assert bbl.workspace_bytes() == 0


@pytest.mark.parametrize("storage,overlap", [("fp64", None), ("fp64", 0), ("fp32", None)])
def test_solve_through_a_deflation_matches_the_dense_spectrum(storage, overlap):
    """H = diag(H1, H2), H1 the 6-point 1-D Laplacian and H2 the 200-point one
    shifted by 1.  Pivot column 0 lives on H1 alone, so the block Krylov
    space exhausts H1's 6-dimensional invariant subspace within a few blocks;
    CholQR2 then deflates a column of W (Sec. II.A, the rank-deficient block)
    and the solver replaces it with a fresh random direction, while the SpMM
    of the next block is already enqueued (it is formed again after the
    replacement).  The lowest 4 eigenvalues are those of the dense matrix."""
    torch, bbl = need_gpu()
    import scipy.sparse as sp
    n1, n2 = 6, 200
    L1 = synth.laplacian_1d(n1)
    L2 = synth.laplacian_1d(n2)
    a1 = sp.csr_matrix((L1.val, L1.col, L1.row_ptr), shape=(n1, n1))
    a2 = sp.csr_matrix((L2.val, L2.col, L2.row_ptr), shape=(n2, n2)) + sp.identity(n2)
    H = synth.csr_from_scipy(sp.block_diag([a1, a2]))
    piv = OR.normal_block(11, H.n, 2)
    piv[n1:, 0] = 0.0
    ref = np.linalg.eigvalsh(sp.block_diag([a1, a2]).toarray())[:4]
    opts = {} if overlap is None else {"ritz_overlap": overlap}
    res = bbl.solve(bbl.Matrix(H, storage=storage, keep_fp64=(storage == "fp32")), 4, 2, pivot=piv, tol=1e-8,
                    check_every=1, **opts)
    assert res.converged
    assert res.stats["deflations"] >= 1
    _check_eigs(res, ref, H, 1e-8)


def test_solve_evecs_into_page_locked_host_memory_and_matrix_from_pinned_csr():
    """A matrix built from page-locked host CSR arrays equals one built from
    numpy arrays, and evecs="pinned" returns the eigenvectors in a
    page-locked CPU tensor equal to the device result."""
    torch, bbl = need_gpu()
    import types
    H = synth.kron_matrix("kron_n2e4", scale=0.3)
    Hp = types.SimpleNamespace(n=H.n, row_ptr=torch.from_numpy(H.row_ptr).pin_memory(),
                               col=torch.from_numpy(H.col).pin_memory(), val=torch.from_numpy(H.val).pin_memory())
    M = bbl.Matrix(H)
    Mp = bbl.Matrix(Hp)
    assert Mp.nnz == M.nnz and Mp.norm_inf == M.norm_inf
    np.testing.assert_array_equal(Mp.diagonal().cpu().numpy(), M.diagonal().cpu().numpy())
    piv = OR.normal_block(5, H.n, 4)
    rd = bbl.solve(M, 4, 4, pivot=piv, tol=1e-8, evecs="device")
    rp = bbl.solve(Mp, 4, 4, pivot=piv, tol=1e-8, evecs="pinned")
    assert rp.evecs.device.type == "cpu" and rp.evecs.is_pinned()
    # the Gram-Schmidt kernels hand out row chunks dynamically: equal up to
    # the order of their partial sums
    np.testing.assert_allclose(rp.evals, rd.evals, rtol=1e-12)
    np.testing.assert_allclose(rp.evecs.numpy(), rd.evecs.cpu().numpy(), atol=1e-9)

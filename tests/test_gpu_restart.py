"""Thick-restart block Lanczos on the GPU (option restart_keep) against the
oracle's block_lanczos_thick and the dense spectrum.

The GPU rotates the kept Ritz vectors so that the projected matrix stays
block tridiagonal (an orthogonal similarity of the oracle's arrowhead), so
the Ritz values agree to rounding; the eigenvalues must match to relative
1e-10, and the number of blocks to convergence agrees with the oracle's to a
few blocks (the convergence tests see slightly different rounding).
"""
import numpy as np
import pytest

import synth
from oracle import lanczos as OL
from oracle import rng as OR
from oracle.spmm import norm_inf, spmm as ospmm
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _lap1d_eigs(n):
    k = np.arange(1, n + 1)
    return np.sort(2.0 - 2.0 * np.cos(k * np.pi / (n + 1)))


@pytest.mark.parametrize("b,keep,mv", [(4, 8, 24), (4, 12, 32), (2, 8, 20), (8, 16, 40)])
def test_restart_fp64_matches_oracle_and_dense(b, keep, mv):
    torch, bbl = need_gpu()
    A = synth.random_sparse_symmetric(300, 6, seed=34)
    nev = 4
    w = np.linalg.eigvalsh(A.to_dense())[:nev]
    piv = OR.normal_block(2, A.n, b)
    ref = OL.block_lanczos_thick(A, nev, b, piv, tol=1e-10, max_vectors=mv, keep=keep)
    res = bbl.solve(bbl.Matrix(A), nev, b, pivot=piv, tol=1e-10, max_vectors=mv, restart_keep=keep, check_every=1)
    assert ref.converged and ref.restarts >= 1
    assert res.converged and res.stats["restarts"] >= 1
    np.testing.assert_allclose(res.evals, w, rtol=1e-10)
    np.testing.assert_allclose(res.evals, ref.evals, rtol=1e-10)
    assert abs(res.stats["iters"] - ref.iters) <= max(3, ref.iters // 10)
    X = res.evecs.cpu().numpy()
    assert np.abs(X.T @ X - np.eye(nev)).max() < 1e-8
    R = ospmm(A, X) - X * res.evals
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-10 * norm_inf(A) * 1.01)


def test_restart_laplacian_closed_form():
    torch, bbl = need_gpu()
    n = 400
    H = synth.laplacian_1d(n)
    res = bbl.solve(bbl.Matrix(H), 3, 2, pivot=OR.normal_block(3, n, 2), tol=1e-10, max_vectors=40, restart_keep=8)
    assert res.converged and res.stats["restarts"] >= 1
    np.testing.assert_allclose(res.evals, _lap1d_eigs(n)[:3], rtol=1e-9)


def test_restart_kron_fp64_and_mixed_precision_match_oracle():
    """The Kronecker workload with a basis far too small to converge without
    restarts: FP64, and FP32 storage whose float-float polish restarts too."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    piv = OR.normal_block(7, H.n, 8)
    ref = OL.block_lanczos(H, 8, 8, piv, tol=1e-9)
    unres = bbl.solve(bbl.Matrix(H), 8, 8, pivot=piv, tol=1e-9, max_vectors=64)
    assert unres.status == "BBL_ERR_NOT_CONVERGED"
    r64 = bbl.solve(bbl.Matrix(H), 8, 8, pivot=piv, tol=1e-9, max_vectors=64, restart_keep=16)
    assert r64.converged and r64.stats["restarts"] >= 1
    np.testing.assert_allclose(r64.evals, ref.evals, rtol=1e-10)
    M32 = bbl.Matrix(H, storage="fp32", fmt="sell", sell_sigma=256)
    r32 = bbl.solve(M32, 8, 8, pivot=piv, tol=1e-9, max_vectors=64, restart_keep=16)
    assert r32.converged and r32.stats["restarts"] >= 1 and r32.stats["polish_iters"] >= 1
    np.testing.assert_allclose(r32.evals, ref.evals, rtol=1e-10)
    X = r32.evecs.cpu().numpy()
    R = ospmm(H, X) - X * r32.evals
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-9 * norm_inf(H) * 1.01)


def test_restart_stops_at_max_blocks_and_rejects_bad_keep():
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.5)
    M = bbl.Matrix(H)
    piv = OR.normal_block(7, H.n, 8)
    r = bbl.solve(M, 8, 8, pivot=piv, tol=1e-13, max_vectors=48, restart_keep=16, max_blocks=25)
    assert r.status == "BBL_ERR_NOT_CONVERGED" and r.stats["iters"] == 25 and r.stats["restarts"] >= 1
    assert np.all(np.isfinite(r.evals))
    for keep in (12, 4, 24):   # not a multiple of b, below nev, above 16
        with pytest.raises(bbl.BBLError):
            bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, max_vectors=48, restart_keep=keep)

"""The Kronecker-factored operator (bbl_matrix_create_kron) against the oracle.

The operator applies H = Hp (x) I + I (x) Hn + sum_k Cp_k (x) Cn_k from its
factors (the paper's on-the-fly matrix elements, Sec. I, Sec. III.A,
Appendix A).  The matrix it applies is the exact Kronecker sum, so the
oracle works on the same workload assembled with unrounded entries
(synth.assemble(..., exact=True)).

Tolerances.  FP64: every output entry is a sum of products of the factor
values and V; the GPU forms sum_e a_e V[p'] then the n-factor product, the
oracle sums the assembled row, so the two differ by rounding only:
|W_gpu - W_ref| <= 64 * eps64 * (sum_t |A_t| (x) |B_t|) |V| entrywise.  FP32
blocks: the same with eps32.  Whole solves: eigenvalues to relative 1e-10.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import lanczos as OL
from oracle import pivot as OP
from oracle import rng as OR
from oracle.spmm import norm_inf, spmm as ospmm, spmm_rows
from tests.gpu_util import need_gpu, principal_angle_sin, to_dev

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _abs_factors(f):
    """The factors with absolute values (for the entrywise rounding bound)."""
    ab = lambda m: synth.CSR(m.n, m.row_ptr, m.col, np.abs(m.val))
    return synth.KronFactors(ab(f.Hp), ab(f.Hn), [ab(x) for x in f.Cp], [ab(x) for x in f.Cn])


def _factors(kind):
    if kind == "small":
        return synth.named_factors("kron_n2e4", scale=0.3)          # 60 x 30, K = 4
    if kind == "ragged":
        return synth.kron_factors(23, 37, 3, 2.5, seed=5)            # odd sizes, sparse couplings
    if kind == "nocoupling":
        return synth.kron_factors(40, 50, 0, 1.0, seed=6)            # K = 0
    if kind == "wide":
        return synth.kron_factors(9, 3000, 2, 3.0, seed=7)           # nN = 3000: narrower column groups, 1024 threads
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["small", "ragged", "nocoupling", "wide"])
@pytest.mark.parametrize("b", [1, 2, 3, 4, 8, 16])
def test_kron_spmm_fp64_matches_oracle(kind, b):
    torch, bbl = need_gpu()
    f = _factors(kind)
    H = synth.assemble(f, exact=True)
    Habs = synth.assemble(_abs_factors(f), exact=True)
    M = bbl.KronMatrix(f, storage="fp64")
    assert M.n == H.n
    V = np.random.default_rng(b).standard_normal((H.n, b))
    W = bbl.spmm(M, to_dev(torch, V)).cpu().numpy()
    bound = 64 * EPS64 * ospmm(Habs, np.abs(V))
    assert np.all(np.abs(W - ospmm(H, V)) <= bound + 1e-300)


@pytest.mark.parametrize("kind", ["small", "ragged", "wide"])
@pytest.mark.parametrize("b", [1, 4, 8, 16])
def test_kron_spmm_fp32_and_fp64_arithmetic(kind, b):
    """FP32 storage: FP32 blocks in FP32 arithmetic (bbl_spmm) and FP64 blocks
    in FP64 arithmetic on the same FP32 factor values (bbl_spmm_f64)."""
    torch, bbl = need_gpu()
    f = _factors(kind)
    H = synth.assemble(f, exact=True)
    Habs = synth.assemble(_abs_factors(f), exact=True)
    M = bbl.KronMatrix(f, storage="fp32")
    V = np.random.default_rng(10 + b).standard_normal((H.n, b)).astype(np.float32).astype(np.float64)
    ref = ospmm(H, V)
    absb = ospmm(Habs, np.abs(V))
    W32 = bbl.spmm(M, to_dev(torch, V, torch.float32)).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(W32 - ref) <= 64 * EPS32 * absb + 1e-30)
    W64 = bbl.spmm_f64(M, to_dev(torch, V)).cpu().numpy()
    assert np.all(np.abs(W64 - ref) <= 64 * EPS64 * absb + 1e-300)


def test_kron_creation_diag_norm_nnz_match_the_expansion():
    """diag(H), ||H||_inf and the nonzero count computed on the device from
    the factors equal those of the assembled exact matrix (the diagonal
    bit for bit: both sum the terms in the same order)."""
    torch, bbl = need_gpu()
    for kind in ("small", "ragged", "nocoupling"):
        f = _factors(kind)
        H = synth.assemble(f, exact=True)
        M = bbl.KronMatrix(f, storage="fp64", check_symmetry=True)
        assert M.nnz == H.nnz
        np.testing.assert_array_equal(M.diagonal().cpu().numpy(), H.diagonal())
        assert M.norm_inf == pytest.approx(norm_inf(H), rel=1e-14)


def test_kron_rejects_bad_factors_on_the_host():
    torch, bbl = need_gpu()
    f = _factors("small")
    bad = synth.KronFactors(f.Hp, f.Hn, list(f.Cp), list(f.Cn))
    c = bad.Cn[0]
    col = c.col.copy()
    col[0] = c.n + 5                       # column out of range
    bad.Cn[0] = synth.CSR(c.n, c.row_ptr, col, c.val)
    with pytest.raises(bbl.BBLError) as e:
        bbl.KronMatrix(bad)
    assert e.value.status == 1
    asym = synth.KronFactors(f.Hp, f.Hn, list(f.Cp), list(f.Cn))
    c = asym.Cp[1]
    val = c.val.copy()
    k = int(np.nonzero(c.col != np.repeat(np.arange(c.n), np.diff(c.row_ptr)))[0][0])
    val[k] += 1.0
    asym.Cp[1] = synth.CSR(c.n, c.row_ptr, c.col, val)
    bbl.KronMatrix(asym)                   # accepted without the check
    with pytest.raises(bbl.BBLError) as e:
        bbl.KronMatrix(asym, check_symmetry=True)
    assert e.value.status == 2


def test_kron_spmm_refuses_a_tile_beyond_shared_memory():
    torch, bbl = need_gpu()
    f = synth.kron_factors(3, 20000, 1, 2.0, seed=8)     # one 20000-row slab per CTA does not fit
    M = bbl.KronMatrix(f, storage="fp32")
    V = torch.zeros((M.n, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(bbl.BBLError) as e:
        bbl.spmm(M, V)
    assert e.value.status == 8


@pytest.mark.parametrize("b", [1, 4, 8])
def test_kron_solve_fp64_matches_oracle(b):
    torch, bbl = need_gpu()
    f = _factors("small")
    H = synth.assemble(f, exact=True)
    piv = OR.normal_block(5, H.n, b)
    ref = OL.block_lanczos(H, 4, b, piv, tol=1e-8)
    res = bbl.solve(bbl.KronMatrix(f, storage="fp64"), 4, b, pivot=piv, tol=1e-8, check_every=1)
    assert res.converged and ref.converged
    np.testing.assert_allclose(res.evals, ref.evals, rtol=1e-10)
    assert abs(res.stats["iters"] - ref.iters) <= 1
    X = res.evecs.cpu().numpy()
    R = ospmm(H, X) - X * res.evals
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-8 * norm_inf(H) * 1.01)


def test_kron_mixed_precision_solve_with_bootstrap_matches_oracle():
    """FP32 factors and blocks, the float-float polish and FP64 residuals on
    the factored operator, from a bootstrapped pivot whose truncated space
    H[S,S] is extracted from the factors; eigenvalues to 1e-10."""
    torch, bbl = need_gpu()
    f = synth.named_factors("kron_n2e4", scale=0.5)
    H = synth.assemble(f, exact=True)
    ref = OL.block_lanczos(H, 8, 8, OR.normal_block(7, H.n, 8), tol=1e-9)
    M = bbl.KronMatrix(f, storage="fp32")
    P = bbl.pivot_bootstrap(M, 800, 8, sub_tol=1e-4)
    res = bbl.solve(M, 8, 8, pivot=P, tol=1e-9)
    assert res.converged and res.stats["polish_iters"] >= 1
    np.testing.assert_allclose(res.evals, ref.evals, rtol=1e-10)
    X = res.evecs.cpu().numpy()
    R = ospmm(H, X) - X * res.evals
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-9 * norm_inf(H) * 1.01)


def test_kron_bootstrap_submatrix_matches_the_oracle():
    """H[S,S] from the factors gives the bootstrapped pivot of the oracle's
    dense truncated solve of the assembled exact matrix: the same rows S and
    the same subspace to the sub-solve's accuracy (residual 1e-11 * ||H[S,S]||
    over the gap to the fifth eigenvalue), as the stored matrix does."""
    torch, bbl = need_gpu()
    f = synth.named_factors("kron_n2e4", scale=0.4)
    H = synth.assemble(f, exact=True)
    Po, S, _ = OP.bootstrap_pivot(H, 600, 4)
    for M in (bbl.KronMatrix(f, storage="fp64"), bbl.Matrix(H)):
        P = bbl.pivot_bootstrap(M, 600, 4, sub_tol=1e-11).cpu().numpy()
        assert set(np.nonzero(np.abs(P).sum(axis=1))[0]) <= set(S.tolist())
        assert principal_angle_sin(np.linalg.qr(P)[0], Po) < 1e-6


def test_kron_fullsize_spmm_sampled_rows():
    """n = 2,000,000 (2000 x 1000 factors, 12 coupling terms): the FP32
    factored SpMM at b = 8, in the launch configuration the solver uses,
    against the oracle's rows of the exact matrix at 2000 sampled rows."""
    torch, bbl = need_gpu()
    f = synth.named_factors("kron_n2e6")
    M = bbl.KronMatrix(f, storage="fp32")
    H = synth.assemble(f, exact=True)
    Habs = synth.assemble(_abs_factors(f), exact=True)
    assert M.nnz == H.nnz and M.norm_inf == pytest.approx(norm_inf(H), rel=1e-14)
    V = np.random.default_rng(3).standard_normal((H.n, 8)).astype(np.float32)
    W = bbl.spmm(M, to_dev(torch, V)).cpu().numpy().astype(np.float64)
    rows = np.sort(np.random.default_rng(4).choice(H.n, 2000, replace=False))
    rows = np.unique(np.concatenate([rows, [0, 999, 1000, H.n - 1]]))
    V64 = V.astype(np.float64)
    ref = spmm_rows(H, V64, rows)
    bound = 64 * EPS32 * spmm_rows(Habs, np.abs(V64), rows)
    assert np.all(np.abs(W[rows] - ref) <= bound)


def test_kron_fullsize_bootstrap_mixed_precision_matches_oracle():
    """The benchmark's step on the factored operator at n = 2,000,000: the
    bootstrapped pivot (20,000 lowest-diagonal rows, H[S,S] from the factors,
    sub-solve to 1e-4), the FP32 stage to 3e-7 with the FP16 first-pass Gram,
    the float-float polish: the eight eigenvalues against the FP64 oracle's
    eigenvalues of the exact matrix to relative 1e-10."""
    import bench
    path = os.path.join(GOLDEN, "kron_n2e6_exact_fp64_oracle_evals.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle eigenvalues for the exact n = 2e6 matrix")
    ref = json.load(open(path))
    torch, bbl = need_gpu()
    M = bbl.KronMatrix(synth.named_factors("kron_n2e6"), storage="fp32")
    assert M.nnz == ref["nnz"] and M.norm_inf == pytest.approx(ref["norm_inf"], rel=1e-14)
    P = bench.headline_pivot(bbl, M)
    r = bench.headline_solve(bbl, M, P, evecs=None)
    assert r.converged
    rel = np.abs(r.evals - np.array(ref["evals"])) / np.abs(ref["evals"])
    print("factored operator, relative eigenvalue errors vs the FP64 oracle:", " ".join(f"{x:.2e}" for x in rel))
    assert rel.max() <= 1e-10, rel
    assert np.all(r.resid <= ref["tol"] * ref["norm_inf"] * 1.01)

"""Step-level parity of the CUDA kernels with the oracle, through the C ABI.

Tolerances (FP64): every entry of a product is a sum of at most a few
hundred terms, so the GPU and the oracle differ only by summation order:
|W_gpu - W_ref| <= 64 * eps64 * (|H| |V|) entrywise (a bound well above the
worst-case gamma_k for k <= 2000 terms is not needed here: rows are short).
FP32 storage: the same bound with eps32 and the FP32-rounded inputs.
"""
import numpy as np
import pytest

import synth
from oracle import lanczos as OL
from oracle import rng as OR
from oracle.spmm import spmm as ospmm
from tests.gpu_util import abs_bound, need_gpu, principal_angle_sin, to_dev

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def _mat(kind):
    if kind == "ragged":
        # empty rows at the end, a long row (row 0 couples to 300 columns), n not a multiple of 32
        return synth.random_sparse_symmetric(1037, 7, seed=11, empty_rows=5, long_row=300)
    if kind == "kron":
        return synth.kron_matrix("kron_n2e4", scale=0.4)
    if kind == "lap2d":
        return synth.laplacian_2d(33, 31)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["ragged", "kron", "lap2d"])
@pytest.mark.parametrize("b", [1, 2, 3, 4, 8, 16])
def test_spmm_csr_fp64(kind, b):
    torch, bbl = need_gpu()
    A = _mat(kind)
    M = bbl.Matrix(A, storage="fp64")
    V = np.random.default_rng(b).standard_normal((A.n, b))
    W = bbl.spmm(M, to_dev(torch, V)).cpu().numpy()
    ref = ospmm(A, V)
    assert np.all(np.abs(W - ref) <= 64 * EPS64 * abs_bound(A, V) + 1e-300)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_spmm_csr_lane_groups(lanes):
    torch, bbl = need_gpu()
    A = _mat("ragged")
    M = bbl.Matrix(A)
    for b in (1, 4, 8, 16):
        V = np.random.default_rng(lanes + b).standard_normal((A.n, b))
        W = bbl.spmm(M, to_dev(torch, V), lanes_per_row=lanes).cpu().numpy()
        ref = ospmm(A, V)
        assert np.all(np.abs(W - ref) <= 64 * EPS64 * abs_bound(A, V) + 1e-300)


@pytest.mark.parametrize("b", [1, 2, 8, 16])
def test_spmm_sell_fp64_storage(b):
    """FP64 values in SELL-C-sigma: 16-byte loads, b*8/16 lanes per row (up
    to 8 for b = 16), against the oracle's product."""
    torch, bbl = need_gpu()
    A = _mat("ragged")
    M = bbl.Matrix(A, storage="fp64", fmt="sell", sell_sigma=64)
    V = np.random.default_rng(30 + b).standard_normal((A.n, b))
    W = bbl.spmm(M, to_dev(torch, V)).cpu().numpy()
    assert np.all(np.abs(W - ospmm(A, V)) <= 64 * EPS64 * abs_bound(A, V))


@pytest.mark.parametrize("fmt,sigma", [("csr", 0), ("sell", 32), ("sell", 256), ("sell", 1024)])
@pytest.mark.parametrize("b", [1, 4, 5, 8, 16])
def test_spmm_fp32_csr_and_sell(fmt, sigma, b):
    torch, bbl = need_gpu()
    A = _mat("ragged")
    M = bbl.Matrix(A, storage="fp32", fmt=fmt, sell_sigma=sigma)
    V32 = np.random.default_rng(b).standard_normal((A.n, b)).astype(np.float32)
    W = bbl.spmm(M, to_dev(torch, V32)).cpu().numpy().astype(np.float64)
    ref = ospmm(A, V32.astype(np.float64))
    assert np.all(np.abs(W - ref) <= 64 * EPS32 * abs_bound(A, V32.astype(np.float64)) + 1e-30)


@pytest.mark.parametrize("fmt", ["csr", "sell"])
def test_spmm_f64_arithmetic_on_fp32_storage(fmt):
    torch, bbl = need_gpu()
    A = _mat("kron")  # FP32-exact values, so FP64 arithmetic reproduces the FP64 product
    M = bbl.Matrix(A, storage="fp32", fmt=fmt, sell_sigma=128)
    V = np.random.default_rng(2).standard_normal((A.n, 8))
    W = bbl.spmm_f64(M, to_dev(torch, V)).cpu().numpy()
    assert np.all(np.abs(W - ospmm(A, V)) <= 64 * EPS64 * abs_bound(A, V))


def test_sell_padding_and_permutation_accounting():
    torch, bbl = need_gpu()
    A = _mat("ragged")
    M = bbl.Matrix(A, storage="fp32", fmt="sell", sell_sigma=256)
    assert M.padded_nnz >= A.nnz and M.nnz == A.nnz
    assert M.norm_inf == pytest.approx(np.abs(A.to_dense()).sum(axis=1).max(), rel=1e-12)
    np.testing.assert_array_equal(M.diagonal().cpu().numpy(), A.diagonal())


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
@pytest.mark.parametrize("b,nb", [(1, 7), (4, 9), (8, 5), (3, 4), (16, 3)])
def test_block_reorth_matches_oracle_cgs2(dtype, b, nb):
    torch, bbl = need_gpu()
    n = 3001
    rng = np.random.default_rng(b * 10 + nb)
    Qf, _ = np.linalg.qr(rng.standard_normal((n, nb * b)))
    W0 = rng.standard_normal((n, b)) + Qf @ rng.standard_normal((nb * b, b))
    npdt = np.float64 if dtype == "fp64" else np.float32
    Qs = Qf.astype(npdt).astype(np.float64)
    W0s = W0.astype(npdt).astype(np.float64)
    basis = np.stack([Qs[:, j * b:(j + 1) * b] for j in range(nb)])
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    Wd = to_dev(torch, W0s, tdt)
    coeff = bbl.block_reorth(to_dev(torch, basis, tdt), Wd, passes=2).cpu().numpy()
    # oracle: the same two classical passes, in FP64
    c1 = Qs.T @ W0s
    W1 = W0s - Qs @ c1
    c2 = Qs.T @ W1
    W2 = W1 - Qs @ c2
    if dtype == "fp64":
        np.testing.assert_allclose(coeff[0], c1, atol=1e-12 * np.abs(c1).max())
        np.testing.assert_allclose(coeff[1], c2, atol=1e-12 * np.abs(c1).max())
        np.testing.assert_allclose(Wd.cpu().numpy(), W2, atol=1e-12 * np.abs(W0s).max())
    else:
        np.testing.assert_allclose(coeff[0], c1, atol=2e-5 * np.abs(c1).max())
        Wg = Wd.cpu().numpy().astype(np.float64)
        # after two passes W is orthogonal to the basis to FP32 accuracy
        assert np.abs(Qs.T @ Wg).max() <= 1e-5 * np.abs(W0s).max()
        np.testing.assert_allclose(Wg, W2, atol=2e-5 * np.abs(W0s).max())


@pytest.mark.parametrize("n,nb", [(1024, 1), (3001, 5), (70_001, 40), (400_003, 3)])
def test_block_gram_f16_matches_fp64_product_of_the_fp16_basis(n, nb):
    """The FP16 first-pass Gram C = Q16^T W (b = 8, tensor cores) against the
    FP64 product of the same FP16 basis and of W as the kernel rounds it:
    per chunk of 1024 rows, W times the power of two that puts the chunk's
    largest |W| in [2^13, 2^14), rounded to FP16 (nearest even), and the
    product scaled back.  Per chunk the tensor core sums 16 exact products
    per step and 64 steps in FP32, chunks in FP64: entrywise
    |C - C_ref| <= 128 eps32 (|Q16|^T |W16|).  The sizes cover one exact
    chunk, a ragged last chunk, many blocks (odd and even counts), and more
    chunks than persistent CTAs (several chunks per CTA from the ticket
    counter).  Against the unrounded W the error stays below 2^-10 of the
    same scale (the first pass only has to remove the bulk)."""
    import ctypes as C
    torch, bbl = need_gpu()
    from paper_2210_15763_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(n + nb)
    Q = (rng.standard_normal((nb, n, 8)) / np.sqrt(n)).astype(np.float16)
    W = rng.standard_normal((n, 8)).astype(np.float32)
    Qd = torch.from_numpy(Q).cuda()
    Wd = torch.from_numpy(W).cuda()
    Cd = torch.empty((nb * 8, 8), dtype=torch.float64, device="cuda")
    st = lib.bbl_block_gram_f16(n, nb, C.c_void_p(Qd.data_ptr()), C.c_void_p(Wd.data_ptr()),
                                C.c_void_p(Cd.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.bbl_last_error()
    Qh = Q.astype(np.float64)
    W16 = np.empty((n, 8))
    for r0 in range(0, n, 1024):
        Wc = W[r0:r0 + 1024]
        mx = float(np.max(np.abs(Wc)))
        ex = int(np.frexp(np.float32(mx))[1]) if mx > 0 else 0
        sc = np.float32(2.0 ** (14 - ex))
        W16[r0:r0 + 1024] = (Wc * sc).astype(np.float16).astype(np.float64) / float(sc)
    got = Cd.cpu().numpy()
    ref = np.concatenate([Qh[j].T @ W16 for j in range(nb)])
    bound = np.concatenate([np.abs(Qh[j]).T @ np.abs(W16) for j in range(nb)])
    assert np.all(np.abs(got - ref) <= 128 * EPS32 * bound)
    Wh = W.astype(np.float64)
    ref32 = np.concatenate([Qh[j].T @ Wh for j in range(nb)])
    assert np.all(np.abs(got - ref32) <= 2.0 ** -10 * bound)


def test_fp16_first_pass_keeps_the_fp32_stage_and_the_result():
    """The FP32 stage with the FP16 first Gram-Schmidt pass (default) and with
    two FP32 passes reach the same eigenvalues; after the polish both agree
    to the FP64 level."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.6)
    M = bbl.Matrix(H, storage="fp32")
    piv = OR.normal_block(9, H.n, 8)
    r1 = bbl.solve(M, 8, 8, pivot=piv, tol=2e-6, polish=0, max_vectors=800, half_first_pass=1)
    r0 = bbl.solve(M, 8, 8, pivot=piv, tol=2e-6, polish=0, max_vectors=800, half_first_pass=0)
    assert r1.converged and r0.converged
    assert abs(r1.stats["iters"] - r0.stats["iters"]) <= 2
    np.testing.assert_allclose(r1.evals, r0.evals, rtol=2e-6)
    p1 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, max_vectors=800, half_first_pass=1)
    p0 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, max_vectors=800, half_first_pass=0)
    assert p1.converged and p0.converged
    np.testing.assert_allclose(p1.evals, p0.evals, rtol=1e-11)


def _split_bound(K):
    """Entrywise bound, relative to sum_k |a_k| |b_k|, of a sum of K products
    formed on the tensor cores from exact three-part BF16 splits of FP32
    operands (six of the nine partial products, dropping at most 2^-23 of
    |a b| each; bounded here by 2^-22) and accumulated in FP32 (K additions,
    each allowed a full FP32 ulp)."""
    return 2.0 ** -22 + 2 * K * EPS32


@pytest.mark.parametrize("n,nb", [(5, 1), (16, 2), (37, 3), (40, 4), (1000, 7), (20_011, 50), (100_003, 99),
                                  (4096, 128), (70_001, 127)])
def test_block_update_gram_matches_fp64_products(n, nb):
    """The fused first update and second Gram (b = 8, tensor cores):
    W1 = W - Q C1 against the FP64 product of the same FP32 basis and of C1
    rounded to FP32, and C2 = Q^T W1 against the FP64 product with the
    kernel's own W1.  The sizes cover fewer rows than one 16-row chunk, an
    exact chunk, ragged last chunks, one and two blocks (no tensor-core
    update; the two newest blocks are FMA products), odd block counts (the
    last block pair of the Gram, or of the tensor-core update, has one
    block) and the largest supported basis (128 blocks)."""
    torch, bbl = need_gpu()
    rng = np.random.default_rng(7 * n + nb)
    Q = (rng.standard_normal((nb, n, 8)) / np.sqrt(n)).astype(np.float32)
    W = rng.standard_normal((n, 8)).astype(np.float32)
    C1 = rng.standard_normal((nb * 8, 8))
    Qd = torch.from_numpy(Q).cuda()
    Wd = torch.from_numpy(W).cuda()
    C2 = bbl.block_update_gram(Qd, Wd, torch.from_numpy(C1).cuda()).cpu().numpy()
    W1 = Wd.cpu().numpy().astype(np.float64)
    Qf = Q.astype(np.float64)
    C1f = C1.astype(np.float32).astype(np.float64)
    Qcat = np.concatenate(list(Qf), axis=1)          # n x m, column 8j + c = block j column c
    ref1 = W.astype(np.float64) - Qcat @ C1f
    S1 = np.abs(Qcat) @ np.abs(C1f)
    m = nb * 8
    assert np.all(np.abs(W1 - ref1) <= _split_bound(m) * S1 + EPS32 * np.abs(ref1))
    ref2 = Qcat.T @ W1
    S2 = np.abs(Qcat).T @ np.abs(W1)
    assert np.all(np.abs(C2 - ref2) <= _split_bound(n) * S2)
    # typical error far below the worst case: a misplaced fragment would show here
    assert np.abs(C2 - ref2).max() <= 1e-5 * S2.max()
    assert np.abs(W1 - ref1).max() <= 1e-5 * S1.max()


def test_block_update_gram_zero_coefficients_leave_w_exact():
    """C1 = 0: the update subtracts exact zeros (W unchanged bit for bit) and
    C2 is the Gram Q^T W."""
    torch, bbl = need_gpu()
    rng = np.random.default_rng(3)
    n, nb = 3001, 9
    Q = rng.standard_normal((nb, n, 8)).astype(np.float32)
    W = rng.standard_normal((n, 8)).astype(np.float32)
    Wd = torch.from_numpy(W).cuda()
    C2 = bbl.block_update_gram(torch.from_numpy(Q).cuda(), Wd, torch.zeros((nb * 8, 8), dtype=torch.float64,
                                                                             device="cuda")).cpu().numpy()
    assert np.array_equal(Wd.cpu().numpy(), W)
    Qcat = np.concatenate(list(Q.astype(np.float64)), axis=1)
    ref = Qcat.T @ W.astype(np.float64)
    assert np.all(np.abs(C2 - ref) <= _split_bound(n) * (np.abs(Qcat).T @ np.abs(W.astype(np.float64))))


def test_block_update_gram_on_an_orthonormal_basis_removes_the_projection():
    """Orthonormal basis and C1 = Q^T W (the FP32 Gram): W1 = W - Q C1 is
    orthogonal to the basis up to FP32 rounding, and C2 = Q^T W1 is that
    rounding-sized remainder, as the second classical pass expects."""
    torch, bbl = need_gpu()
    rng = np.random.default_rng(5)
    n, nb = 50_001, 40
    Qo, _ = np.linalg.qr(rng.standard_normal((n, nb * 8)))
    Q = np.stack([Qo[:, 8 * j:8 * j + 8] for j in range(nb)]).astype(np.float32)
    W = rng.standard_normal((n, 8)).astype(np.float32)
    Qd = torch.from_numpy(Q).cuda()
    C1 = bbl.block_gram(Qd, torch.from_numpy(W).cuda())
    Wd = torch.from_numpy(W).cuda()
    C2 = bbl.block_update_gram(Qd, Wd, C1).cpu().numpy()
    W1 = Wd.cpu().numpy().astype(np.float64)
    Qcat = np.concatenate(list(Q.astype(np.float64)), axis=1)
    ref1 = W.astype(np.float64) - Qcat @ C1.cpu().numpy().astype(np.float32).astype(np.float64)
    scale = np.abs(W).max()
    assert np.abs(W1 - ref1).max() <= 1e-6 * scale
    assert np.abs(Qcat.T @ W1).max() <= 1e-5 * scale
    np.testing.assert_allclose(C2, Qcat.T @ W1, atol=1e-6 * scale)


def _f16old_coefficients(C, js):
    """The coefficients the FP16-copy update applies: rows of the js older
    blocks times s = 2^(14 - e) (max |C_old| = f 2^e, f in [0.5, 1), e at
    least -100), rounded to FP16 and divided by s; the newer rows rounded to
    FP32."""
    Ce = C.astype(np.float32).astype(np.float64)
    if js > 0:
        mx = np.abs(C[:8 * js]).max()
        s = 2.0 ** (14 - max(int(np.frexp(mx)[1]), -100)) if mx > 0 else 1.0
        Ce[:8 * js] = (C[:8 * js] * s).astype(np.float32).astype(np.float16).astype(np.float64) / s
    return Ce


@pytest.mark.parametrize("n,nb,nnew", [(5, 1, 2), (37, 3, 2), (1000, 7, 2), (20_011, 50, 2), (4096, 9, 0),
                                      (3001, 6, 6), (100_003, 99, 2), (17, 4, 1)])
def test_block_update_f16old_matches_fp64_product(n, nb, nnew):
    """W -= Q C with the blocks older than the nnew newest read from the FP16
    copy (tensor cores, their coefficients scaled by a power of two and
    rounded to FP16): against the FP64 product of exactly those operands,
    within the FP32 sums' rounding.  The sizes cover one block, a ragged
    last 16-row tile, fewer rows than one tile, odd older-block counts (the
    last pair has one block), all blocks FP16 (nnew = 0) and all FP32."""
    torch, bbl = need_gpu()
    rng = np.random.default_rng(11 * n + nb)
    Q = (rng.standard_normal((nb, n, 8)) / np.sqrt(n)).astype(np.float32)
    Q16 = Q.astype(np.float16)
    W = rng.standard_normal((n, 8)).astype(np.float32)
    C = rng.standard_normal((nb * 8, 8))
    Wd = torch.from_numpy(W).cuda()
    bbl.block_update_f16old(torch.from_numpy(Q16).cuda(), torch.from_numpy(Q).cuda(), Wd, torch.from_numpy(C).cuda(),
                            nnew=nnew)
    W1 = Wd.cpu().numpy().astype(np.float64)
    js = max(nb - nnew, 0)
    Qused = np.concatenate([Q16[:js].astype(np.float64), Q[js:].astype(np.float64)], axis=0)
    Qcat = np.concatenate(list(Qused), axis=1)   # n x m
    Ce = _f16old_coefficients(C, js)
    ref = W.astype(np.float64) - Qcat @ Ce
    S = np.abs(Qcat) @ np.abs(Ce)
    m = nb * 8
    assert np.all(np.abs(W1 - ref) <= 2 * (m + 1) * EPS32 * (S + np.abs(W)))
    # the typical error is far below that bound: a misread block would show here
    assert np.abs(W1 - ref).max() <= 1e-5 * (S.max() + np.abs(W).max())


def test_narrow_old_updates_keeps_the_fp32_stage_and_the_result():
    """The FP32 stage with both updates' older blocks read from the FP16 copy
    (default) and from the FP32 basis: the same block counts to within two,
    the FP32-stage eigenvalues to the stage's accuracy, and after the polish
    the same eigenvalues to the FP64 level."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.6)
    M = bbl.Matrix(H, storage="fp32")
    piv = OR.normal_block(13, H.n, 8)
    r1 = bbl.solve(M, 8, 8, pivot=piv, tol=2e-6, polish=0, max_vectors=800, narrow_old_updates=1)
    r0 = bbl.solve(M, 8, 8, pivot=piv, tol=2e-6, polish=0, max_vectors=800, narrow_old_updates=0)
    assert r1.converged and r0.converged
    assert abs(r1.stats["iters"] - r0.stats["iters"]) <= 2
    np.testing.assert_allclose(r1.evals, r0.evals, rtol=2e-6)
    p1 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, max_vectors=800, narrow_old_updates=1)
    p0 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, max_vectors=800, narrow_old_updates=0)
    assert p1.converged and p0.converged
    np.testing.assert_allclose(p1.evals, p0.evals, rtol=1e-11)


def test_fused_update_gram_keeps_the_fp32_stage_and_the_result():
    """The FP32 stage with the fused first update + second Gram and
    with the two FP32-pipe kernels reach the same eigenvalues; after the
    polish both agree to the FP64 level."""
    torch, bbl = need_gpu()
    H = synth.kron_matrix("kron_n2e4", scale=0.6)
    M = bbl.Matrix(H, storage="fp32")
    piv = OR.normal_block(9, H.n, 8)
    r1 = bbl.solve(M, 8, 8, pivot=piv, tol=2e-6, polish=0, max_vectors=800, fused_update_gram=1)
    r0 = bbl.solve(M, 8, 8, pivot=piv, tol=2e-6, polish=0, max_vectors=800, fused_update_gram=0)
    assert r1.converged and r0.converged
    assert abs(r1.stats["iters"] - r0.stats["iters"]) <= 2
    np.testing.assert_allclose(r1.evals, r0.evals, rtol=2e-6)
    p1 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, max_vectors=800, fused_update_gram=1)
    p0 = bbl.solve(M, 8, 8, pivot=piv, tol=1e-9, max_vectors=800, fused_update_gram=0)
    assert p1.converged and p0.converged
    np.testing.assert_allclose(p1.evals, p0.evals, rtol=1e-11)


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
@pytest.mark.parametrize("b", [1, 2, 4, 6, 8, 16])
def test_cholqr2_matches_oracle(dtype, b):
    torch, bbl = need_gpu()
    n = 4099
    W = np.random.default_rng(b).standard_normal((n, b)) * np.linspace(1, 3, b)
    npdt = np.float64 if dtype == "fp64" else np.float32
    Ws = W.astype(npdt).astype(np.float64)
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    Wd = to_dev(torch, Ws, tdt)
    B, nd = bbl.cholqr2(Wd)
    Q = Wd.cpu().numpy().astype(np.float64)
    B = B.cpu().numpy()
    Qo, Bo, d = OL.cholqr2(Ws, 0.0)
    assert nd == 0 and not d
    tol = 1e-12 if dtype == "fp64" else 2e-6
    np.testing.assert_allclose(B, Bo, atol=tol * np.abs(Bo).max())
    np.testing.assert_allclose(Q, Qo, atol=tol * 10)
    assert np.abs(Q.T @ Q - np.eye(b)).max() < (1e-13 if dtype == "fp64" else 2e-6)
    assert np.allclose(np.tril(B, -1), 0.0)


def test_cholqr2_deflates_dependent_column():
    torch, bbl = need_gpu()
    n = 2000
    W = np.random.default_rng(3).standard_normal((n, 4))
    W[:, 2] = W[:, 0] - 2.0 * W[:, 1]
    Wd = to_dev(torch, W)
    B, nd = bbl.cholqr2(Wd, defl_abs=1e-3)
    Q = Wd.cpu().numpy()
    B = B.cpu().numpy()
    assert nd == 1
    assert np.all(Q[:, 2] == 0.0) and np.all(B[2] == 0.0)
    keep = [0, 1, 3]
    assert np.abs(Q[:, keep].T @ Q[:, keep] - np.eye(3)).max() < 1e-13
    np.testing.assert_allclose(Q @ B, W, atol=1e-10)


def _band(T, p):
    m = T.shape[0]
    Tb = np.zeros((m, p + 1))
    for i in range(m):
        for d in range(p + 1):
            if i - d >= 0:
                Tb[i, d] = T[i, i - d]
    return Tb


def _random_band(m, p, seed):
    rng = np.random.default_rng(seed)
    T = np.zeros((m, m))
    for d in range(p + 1):
        v = rng.standard_normal(m - d)
        T += np.diag(v, -d)
        if d:
            T += np.diag(v, d)
    return T


@pytest.mark.parametrize("m,p,nev", [(8, 4, 4), (64, 1, 5), (200, 4, 8), (333, 8, 8), (512, 16, 12), (1200, 8, 8)])
def test_ritz_banded_random(m, p, nev):
    torch, bbl = need_gpu()
    T = _random_band(m, p, m + p)
    w, U = np.linalg.eigh(T)
    th, S = bbl.ritz_banded(to_dev(torch, _band(T, p)), nev)
    th = th.cpu().numpy()
    S = S.cpu().numpy()
    scale = np.abs(w).max()
    np.testing.assert_allclose(th, w[:nev], atol=1e-12 * scale)
    assert np.abs(S.T @ S - np.eye(nev)).max() < 1e-10
    assert np.abs(T @ S - S * th).max() < 1e-10 * scale
    for i in range(nev):  # sign convention: first largest-magnitude entry positive
        k = int(np.argmax(np.abs(S[:, i])))
        assert S[k, i] > 0


def test_ritz_banded_degenerate_clusters():
    # block-diagonal T with repeated blocks: every eigenvalue has multiplicity 3
    torch, bbl = need_gpu()
    blk = _random_band(40, 3, 5)
    T = np.kron(np.eye(3), blk)
    p = 3
    w = np.linalg.eigvalsh(T)
    th, S = bbl.ritz_banded(to_dev(torch, _band(T, p)), 9)
    th = th.cpu().numpy()
    S = S.cpu().numpy()
    np.testing.assert_allclose(th, w[:9], atol=1e-11 * np.abs(w).max())
    assert np.abs(S.T @ S - np.eye(9)).max() < 1e-9
    assert np.abs(T @ S - S * th).max() < 1e-9 * np.abs(w).max()


def test_ritz_banded_from_lanczos_T_of_2d_laplacian():
    # the T that the oracle's block Lanczos builds on a 2-D Laplacian (double eigenvalues)
    torch, bbl = need_gpu()
    H = synth.laplacian_2d(20, 20)
    r = OL.block_lanczos(H, 6, 4, OR.normal_block(1, H.n, 4), tol=1e-30, max_vectors=120)
    T = r.T
    w = np.linalg.eigvalsh(T)
    th, S = bbl.ritz_banded(to_dev(torch, _band(T, 4)), 6)
    np.testing.assert_allclose(th.cpu().numpy(), w[:6], atol=1e-12 * np.abs(w).max())


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
@pytest.mark.parametrize("b,nb,k", [(4, 6, 4), (8, 3, 8), (3, 5, 2), (16, 2, 16), (1, 9, 3)])
def test_ritz_vectors_match_basis_times_S(dtype, b, nb, k):
    torch, bbl = need_gpu()
    n = 2777
    rng = np.random.default_rng(b + nb + k)
    npdt = np.float64 if dtype == "fp64" else np.float32
    Q = rng.standard_normal((nb, n, b)).astype(npdt)
    S = rng.standard_normal((nb * b, k))
    tdt = torch.float64 if dtype == "fp64" else torch.float32
    X = bbl.ritz_vectors(to_dev(torch, Q, tdt), to_dev(torch, S)).cpu().numpy()
    Qf = np.concatenate([Q[j].astype(np.float64) for j in range(nb)], axis=1)
    ref = Qf @ S
    bound = np.abs(Qf) @ np.abs(S)
    if dtype == "fp64":
        assert np.all(np.abs(X - ref) <= 64 * EPS64 * bound + 1e-300)
    else:
        # FP32 products summed in FP32 within 256-column tiles, FP64 across
        assert np.all(np.abs(X - ref) <= 258 * 2.0 ** -24 * bound + 1e-300)


def test_pivot_random_is_the_published_generator():
    torch, bbl = need_gpu()
    P = bbl.pivot_random(1000, 4, seed=77).cpu().numpy()
    np.testing.assert_allclose(P, OR.normal_block(77, 1000, 4), rtol=1e-13, atol=1e-13)

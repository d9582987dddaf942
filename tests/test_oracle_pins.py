"""Pins of the CPU oracle against facts fixed by mathematics and the paper.

None of these compares the oracle with itself: they use closed-form spectra,
brute-force dense eigensolves, invariants of the Lanczos recurrence, special
cases of the method (b = 1, an exact pivot, a symmetry-sector pivot) and
published reference values.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import lanczos as L
from oracle import mlp as M
from oracle import pivot as P
from oracle import pivot as P_
from oracle import rng as R
from oracle.spmm import norm_inf, spmm, spmm_loops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lap1d_eigs(n):
    k = np.arange(1, n + 1)
    return np.sort(2.0 - 2.0 * np.cos(k * np.pi / (n + 1)))


def lap1d_vec(n, k):
    i = np.arange(1, n + 1)
    return math.sqrt(2.0 / (n + 1)) * np.sin(i * k * np.pi / (n + 1))


# ----------------------------------------------------------------- rng
def test_splitmix64_reference_values():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    got = [int(x) for x in R.splitmix64(0, np.arange(3, dtype=np.uint64))]
    assert got == want


def test_normal_block_moments():
    z = R.normal_block(7, 20000, 4)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


# ----------------------------------------------------------------- spmm (Eq. 3)
@pytest.mark.parametrize("b", [1, 3, 8])
def test_spmm_matches_definition_and_dense(b):
    A = synth.random_sparse_symmetric(37, 5, seed=3, empty_rows=3, long_row=20)
    V = np.random.default_rng(1).standard_normal((A.n, b))
    W_loop = spmm_loops(A.row_ptr, A.col, A.val, V)
    W_dense = A.to_dense() @ V
    np.testing.assert_allclose(W_loop, W_dense, rtol=0, atol=1e-12)
    np.testing.assert_allclose(spmm(A, V), W_dense, rtol=0, atol=1e-12)


def test_norm_inf_is_max_abs_row_sum():
    A = synth.random_sparse_symmetric(30, 4, seed=5)
    assert norm_inf(A) == pytest.approx(np.abs(A.to_dense()).sum(axis=1).max(), rel=1e-15)


# ----------------------------------------------------------------- closed forms
def test_vector_lanczos_laplacian_1d_closed_form():
    n = 120
    H = synth.laplacian_1d(n)
    v1 = R.normal_block(11, n, 1)[:, 0]
    r = L.vector_lanczos(H, v1, nev=3, tol=1e-10, max_iter=n)
    assert r.converged
    np.testing.assert_allclose(r.evals, lap1d_eigs(n)[:3], rtol=1e-10, atol=1e-13)
    for k in range(3):
        v = lap1d_vec(n, k + 1)
        assert abs(abs(v @ r.evecs[:, k]) - 1.0) < 1e-8


@pytest.mark.parametrize("normaliser", ["cholqr2", "spectral"])
def test_block_lanczos_laplacian_1d_closed_form(normaliser):
    n = 150
    H = synth.laplacian_1d(n)
    r = L.block_lanczos(H, 4, 2, R.normal_block(5, n, 2), tol=1e-10, normaliser=normaliser)
    assert r.converged
    np.testing.assert_allclose(r.evals, lap1d_eigs(n)[:4], rtol=1e-10, atol=1e-13)
    assert np.all(r.resid <= 1e-9 * norm_inf(H))


def test_block_lanczos_laplacian_2d_multiplicities():
    nx = ny = 16
    H = synth.laplacian_2d(nx, ny)
    e1 = lap1d_eigs(nx)
    want = np.sort((e1[:, None] + e1[None, :]).ravel())[:6]
    assert want[1] == pytest.approx(want[2])  # lambda_(1,2) = lambda_(2,1): a double eigenvalue
    r = L.block_lanczos(H, 6, 4, R.normal_block(2, H.n, 4), tol=1e-10)
    assert r.converged
    np.testing.assert_allclose(r.evals, want, rtol=1e-10, atol=1e-12)


def test_kronecker_without_coupling_is_sum_of_factor_spectra():
    f = synth.kron_factors(30, 20, K=0, c=3.0, seed=9)
    # factor values on a 2^-12 grid so that every assembled sum is exact in FP32
    for F in (f.Hp, f.Hn):
        F.val = np.round(F.val * 4096.0) / 4096.0
    H = synth.assemble(f)
    ep = np.linalg.eigvalsh(f.Hp.to_dense())
    en = np.linalg.eigvalsh(f.Hn.to_dense())
    want = np.sort((ep[:, None] + en[None, :]).ravel())[:4]
    r = L.block_lanczos(H, 4, 4, R.normal_block(1, H.n, 4), tol=1e-10)
    np.testing.assert_allclose(r.evals, want, rtol=1e-10, atol=1e-11)


# ----------------------------------------------------------------- brute force
@pytest.mark.parametrize("b", [1, 3, 5])
def test_block_lanczos_vs_dense_eigensolve(b):
    A = synth.random_sparse_symmetric(90, 6, seed=b)
    want = np.linalg.eigvalsh(A.to_dense())[:5]
    r = L.block_lanczos(A, 5, b, R.normal_block(3, A.n, b), tol=1e-11, max_vectors=90)
    np.testing.assert_allclose(r.evals, want, rtol=1e-10, atol=1e-11)


def test_kron_small_vs_dense():
    H = synth.kron_matrix("kron_n2e4", scale=0.1)
    want = np.linalg.eigvalsh(H.to_dense())[:4]
    r = L.block_lanczos(H, 4, 4, R.normal_block(4, H.n, 4), tol=1e-10)
    assert r.converged
    np.testing.assert_allclose(r.evals, want, rtol=1e-10)


# ----------------------------------------------------------------- b = 1 is Algorithm 1
def test_block_b1_reproduces_vector_lanczos():
    A = synth.random_sparse_symmetric(200, 6, seed=21)
    v1 = R.normal_block(8, A.n, 1)
    rv = L.vector_lanczos(A, v1[:, 0], nev=2, tol=1e-30, max_iter=25)
    rb = L.block_lanczos(A, 2, 1, v1, tol=1e-30, max_vectors=25)
    alpha_v = np.array([a[0, 0] for a in rv.A])
    alpha_b = np.array([a[0, 0] for a in rb.A])
    beta_v = np.array([x[0, 0] for x in rv.B])
    beta_b = np.array([x[0, 0] for x in rb.B])
    np.testing.assert_allclose(alpha_b, alpha_v, rtol=0, atol=1e-12 * norm_inf(A))
    np.testing.assert_allclose(np.abs(beta_b), np.abs(beta_v), rtol=0, atol=1e-12 * norm_inf(A))


# ----------------------------------------------------------------- invariants
def test_invariants_orthonormality_projection_interlacing():
    H = synth.kron_matrix("kron_n2e4", scale=0.15)
    b = 3
    r = L.block_lanczos(H, 4, b, R.normal_block(6, H.n, b), tol=1e-9, keep_basis=True)
    V = r.V
    m = V.shape[1]
    assert np.max(np.abs(V.T @ V - np.eye(m))) < 1e-12
    HV = spmm(H, V)
    assert np.max(np.abs(V.T @ HV - r.T)) < 1e-11 * norm_inf(H)
    # Cauchy interlacing: the i-th Ritz value never increases as the space grows
    for j in range(1, len(r.theta_history)):
        prev, cur = r.theta_history[j - 1], r.theta_history[j]
        k = min(4, prev.size)
        assert np.all(cur[:k] <= prev[:k] + 1e-10 * norm_inf(H))
    # and stays above the true eigenvalue
    want = np.linalg.eigvalsh(H.to_dense())[:4]
    assert np.all(r.theta_history[-1][:4] >= want - 1e-9)
    # residual estimate ||B_j s_i[last b]|| equals the true residual up to round-off
    np.testing.assert_allclose(r.resid, r.resid_est, rtol=1e-3, atol=1e-12 * norm_inf(H))


def test_spectral_and_cholqr2_give_the_same_ritz_values():
    H = synth.kron_matrix("kron_n2e4", scale=0.2)
    piv = R.normal_block(12, H.n, 4)
    a = L.block_lanczos(H, 4, 4, piv, tol=1e-30, max_vectors=60, normaliser="cholqr2")
    c = L.block_lanczos(H, 4, 4, piv, tol=1e-30, max_vectors=60, normaliser="spectral")
    np.testing.assert_allclose(a.theta_history[-1][:8], c.theta_history[-1][:8], rtol=1e-12)


# ----------------------------------------------------------------- normalisers
def test_cholqr2_matches_householder_qr():
    W = np.random.default_rng(3).standard_normal((500, 6))
    Q, B, d = L.cholqr2(W, 0.0)
    assert not d
    assert np.max(np.abs(Q.T @ Q - np.eye(6))) < 1e-14
    np.testing.assert_allclose(Q @ B, W, atol=1e-13)
    q, r = np.linalg.qr(W)
    s = np.sign(np.diag(r))
    np.testing.assert_allclose(B, s[:, None] * r, atol=1e-12)
    assert np.allclose(np.tril(B, -1), 0.0)


def test_cholqr2_deflates_dependent_column():
    rng = np.random.default_rng(4)
    basis, _ = np.linalg.qr(rng.standard_normal((300, 5)))
    W = rng.standard_normal((300, 4))
    W -= basis @ (basis.T @ W)
    W[:, 2] = 2.0 * W[:, 0] - W[:, 1]          # exactly dependent column
    Q, B, d = L.cholqr2(W, 1e-20, basis, lambda i: L.deflation_vector(0, 1, i, 300))
    assert d == [2]
    assert np.max(np.abs(Q.T @ Q - np.eye(4))) < 1e-13
    assert np.max(np.abs(basis.T @ Q)) < 1e-13
    np.testing.assert_allclose(Q @ B, W, atol=1e-12)
    assert np.allclose(np.tril(B, -1), 0.0)


def test_spectral_normalise_deflates_dependent_column():
    """Eqs. 9-11 with a near-singular overlap (Sec. II.B: such directions are
    removed): an exactly dependent column of W' gives one zero eigenvalue of
    O = W'^T W'; its row of B is zero, its column of V_{n+1} is a unit vector
    orthogonal to the basis and to the kept columns, and V_{n+1} B = W' still
    holds because W' has no component along the removed direction."""
    rng = np.random.default_rng(4)
    basis, _ = np.linalg.qr(rng.standard_normal((300, 5)))
    W = rng.standard_normal((300, 4))
    W -= basis @ (basis.T @ W)
    W[:, 2] = 2.0 * W[:, 0] - W[:, 1]          # exactly dependent column
    V, B, removed = L.spectral_normalise(W, 1e-20, basis, lambda i: L.deflation_vector(0, 1, i, 300))
    assert removed == [0]                      # eigh orders the overlap's eigenvalues ascending
    assert np.max(np.abs(V.T @ V - np.eye(4))) < 1e-13
    assert np.max(np.abs(basis.T @ V)) < 1e-13
    assert np.all(B[0] == 0.0)
    np.testing.assert_allclose(V @ B, W, atol=1e-12)
    np.testing.assert_allclose(B.T @ B, W.T @ W, atol=1e-11)   # Eq. 10 read as Lambda^{1/2} U^T
    # the kept columns span exactly the column space of W'
    P = V[:, 1:] @ V[:, 1:].T
    np.testing.assert_allclose(P @ W, W, atol=1e-12)


@pytest.mark.parametrize("normaliser", ["spectral", "cholqr2"])
def test_block_lanczos_deflation_branch_reaches_the_dense_spectrum(normaliser):
    """A pivot holding an exact eigenvector: its column of W' vanishes after
    the reorthogonalisation of the first block, so both normalisers take
    their deflation branch there (a replacement direction enters the Krylov
    space), and both still converge to the dense eigenvalues."""
    A = synth.random_sparse_symmetric(150, 6, seed=21)
    w, U = np.linalg.eigh(A.to_dense())
    piv = R.normal_block(8, A.n, 4)
    piv[:, 0] = U[:, 0]
    r = L.block_lanczos(A, 4, 4, piv, tol=1e-11, max_vectors=150, normaliser=normaliser)
    assert r.deflations >= 1
    assert r.converged
    np.testing.assert_allclose(r.evals, w[:4], rtol=1e-10)
    # with a deflation the method has the same Ritz values under either normaliser
    other = L.block_lanczos(A, 4, 4, piv, tol=1e-11, max_vectors=150,
                            normaliser="cholqr2" if normaliser == "spectral" else "spectral")
    np.testing.assert_allclose(r.evals, other.evals, rtol=1e-10)


# ----------------------------------------------------------------- thick restart
def test_thick_restart_off_is_block_lanczos():
    A = synth.random_sparse_symmetric(300, 6, seed=33)
    piv = R.normal_block(1, A.n, 4)
    a = L.block_lanczos(A, 4, 4, piv, tol=1e-10)
    t = L.block_lanczos_thick(A, 4, 4, piv, tol=1e-10, keep=0)
    assert t.iters == a.iters and t.restarts == 0
    np.testing.assert_allclose(t.evals, a.evals, rtol=1e-13)


@pytest.mark.parametrize("b,keep,mv", [(4, 8, 24), (4, 12, 32), (2, 6, 16), (1, 4, 10)])
def test_thick_restart_reaches_the_dense_spectrum(b, keep, mv):
    A = synth.random_sparse_symmetric(300, 6, seed=34)
    w = np.linalg.eigvalsh(A.to_dense())[:4]
    r = L.block_lanczos_thick(A, 4, b, R.normal_block(2, A.n, b), tol=1e-10, max_vectors=mv, keep=keep)
    assert r.converged and r.restarts >= 1
    np.testing.assert_allclose(r.evals, w, rtol=1e-10)
    assert np.all(r.resid <= 1e-10 * norm_inf(A) * 1.01)


def test_thick_restart_laplacian_closed_form():
    n = 400
    H = synth.laplacian_1d(n)
    r = L.block_lanczos_thick(H, 3, 2, R.normal_block(3, n, 2), tol=1e-10, max_vectors=40, keep=8, max_blocks=20000)
    assert r.converged and r.restarts >= 1
    np.testing.assert_allclose(r.evals, lap1d_eigs(n)[:3], rtol=1e-9)


def test_thick_restart_keeps_an_orthonormal_basis_and_its_projection():
    """After restarts the stored basis Q = [X, V_0, ...] is orthonormal and
    Q^T H Q is the arrowhead-plus-Eq.-12 matrix the method solves."""
    A = synth.kron_matrix("kron_n2e4", scale=0.3)
    r = L.block_lanczos_thick(A, 4, 4, R.normal_block(4, A.n, 4), tol=1e-30, max_vectors=40, keep=8,
                              max_blocks=30, keep_basis=True)
    assert r.restarts >= 2
    Q = r.V
    assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-12
    np.testing.assert_allclose(Q.T @ spmm(A, Q), r.T, atol=1e-9 * norm_inf(A))


def test_thick_restart_ritz_values_never_increase():
    """The kept Ritz vectors span a subspace of every later basis, so by the
    minimax principle each of the lowest Ritz values can only decrease."""
    A = synth.random_sparse_symmetric(300, 6, seed=35)
    r = L.block_lanczos_thick(A, 4, 4, R.normal_block(5, A.n, 4), tol=1e-12, max_vectors=24, keep=8)
    assert r.restarts >= 2
    low = np.array([h[:4] for h in r.theta_history if h.size >= 4])
    assert np.all(np.diff(low, axis=0) <= 1e-12 * norm_inf(A))


def test_block_tridiagonal_layout():
    A = [np.full((2, 2), 1.0), np.full((2, 2), 2.0)]
    B = [np.array([[3.0, 4.0], [0.0, 5.0]])]
    T = L.block_tridiagonal(A, B)
    assert T[2, 0] == 3.0 and T[2, 1] == 4.0 and T[3, 1] == 5.0 and T[3, 0] == 0.0
    np.testing.assert_array_equal(T, T.T)


# ----------------------------------------------------------------- method special cases
def test_exact_pivot_converges_in_one_block():
    A = synth.random_sparse_symmetric(120, 6, seed=33)
    w, U = np.linalg.eigh(A.to_dense())
    r = L.block_lanczos(A, 4, 4, U[:, :4], tol=1e-10)
    assert r.iters == 1 and r.converged
    np.testing.assert_allclose(r.evals, w[:4], rtol=1e-12)


def test_symmetry_sector_pivot_misses_the_other_sector():
    # H = A + J A J (J the index reversal) commutes with J, so every
    # eigenvector is even or odd.  A pivot in the even sector only builds even
    # Krylov vectors: the lowest (odd) state is an 'intruder' the space lacks
    # (Sec. II.B), while a generic pivot finds it.  Expected values: dense
    # eigensolve split by parity.
    import scipy.sparse as sp
    n = 120
    A = synth.random_sparse_symmetric(n, 6, seed=5).to_scipy()
    J = sp.csr_matrix((np.ones(n), (np.arange(n), np.arange(n)[::-1])), shape=(n, n))
    H = synth.csr_from_scipy(A + J @ A @ J)
    w, U = np.linalg.eigh(H.to_dense())
    parity = np.sign(np.sum(U * U[::-1], axis=0))
    assert parity[0] < 0
    p = R.normal_block(3, n, 2)
    even = 0.5 * (p + p[::-1])
    r = L.block_lanczos(H, 3, 2, even, tol=1e-9, max_vectors=60)
    assert r.converged
    np.testing.assert_allclose(r.evals, w[parity > 0][:3], rtol=1e-10)
    assert r.evals[0] > w[0] + 0.5 * (w[1] - w[0])          # the odd ground state is absent
    mixed = L.block_lanczos(H, 3, 2, p, tol=1e-9, max_vectors=n)
    np.testing.assert_allclose(mixed.evals, w[:3], rtol=1e-10)


def test_bootstrap_pivot_on_full_space_is_exact():
    A = synth.random_sparse_symmetric(80, 5, seed=2)
    piv, S, th = P.bootstrap_pivot(A, A.n, 3)
    w = np.linalg.eigvalsh(A.to_dense())
    np.testing.assert_allclose(th, w[:3], rtol=1e-12)
    r = L.block_lanczos(A, 3, 3, piv, tol=1e-10)
    assert r.iters == 1


def test_pivot_overlap_closed_forms():
    """The overlap of a unit vector with span(P): 1 inside, 0 orthogonal, and
    cos(t) for a pivot column cos(t) x + sin(t) y with y orthogonal to x; a
    dependent pivot column changes nothing; scaling P changes nothing."""
    rng = np.random.default_rng(9)
    Qf, _ = np.linalg.qr(rng.standard_normal((200, 6)))
    x, y, z, w = Qf[:, 0], Qf[:, 1], Qf[:, 2], Qf[:, 3]
    t = 0.3
    P = np.stack([np.cos(t) * x + np.sin(t) * y, z, 2.0 * z + 0.0 * x], axis=1) * 7.0
    o = P_.pivot_overlap(P, np.stack([x, y, z, w], axis=1))
    np.testing.assert_allclose(o, [np.cos(t), np.sin(t), 1.0, 0.0], atol=1e-12)


def test_pivot_overlap_flags_the_missing_symmetry_sector():
    """The paper's intruder case: an even-sector pivot has no overlap with the
    odd-sector eigenvectors (their overlap is zero to rounding) and a
    positive one with the even-sector eigenvectors."""
    import scipy.sparse as sp
    n = 120
    A = synth.random_sparse_symmetric(n, 6, seed=5).to_scipy()
    J = sp.csr_matrix((np.ones(n), (np.arange(n), np.arange(n)[::-1])), shape=(n, n))
    H = (A + J @ A @ J).toarray()
    w, U = np.linalg.eigh(H)
    parity = np.sign(np.sum(U * U[::-1], axis=0))
    p = R.normal_block(3, n, 2)
    even = 0.5 * (p + p[::-1])
    o = P_.pivot_overlap(even, U[:, :6])
    assert np.all(o[parity[:6] < 0] < 1e-12)
    assert np.all(o[parity[:6] > 0] > 1e-3)


def test_truncated_set_ties_take_lower_index():
    d = np.array([3.0, 1.0, 2.0, 1.0, 2.0, 0.5])
    # brute force: sort (value, index) pairs
    want = sorted(sorted(range(d.size), key=lambda i: (d[i], i))[:4])
    assert list(P.truncated_set(d, 4)) == want == [1, 2, 3, 5]


def test_bootstrap_pivot_reduces_iterations_on_diagonally_dominant_matrix():
    # Paper Sec. III: a pivot with good overlap cuts the number of iterations.
    H = synth.kron_matrix("kron_n2e4", scale=0.25)
    b = 4
    rnd = L.block_lanczos(H, 4, b, P.random_pivot(H.n, b, 1), tol=1e-8)
    piv, _, _ = P.bootstrap_pivot(H, H.n // 4, b)
    bst = L.block_lanczos(H, 4, b, piv, tol=1e-8)
    np.testing.assert_allclose(bst.evals, rnd.evals, rtol=1e-10)
    assert bst.iters <= rnd.iters


# ----------------------------------------------------------------- MLP
def test_bf16_round_reference_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1.0 + 2 ** -7], dtype=np.float32)
    got = M.bf16_round(x)
    # 1+2^-8 is a tie -> even (1.0); 1+3*2^-8 is a tie -> even (1+2^-6); 1+2^-7 is representable
    np.testing.assert_array_equal(got, [1.0, 1.0, 1.0 + 2 ** -6, -2.5, 1.0 + 2 ** -7])


def test_gelu_closed_forms():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert M.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5)
    x = np.array([1.0])
    assert M.gelu(x)[0] == pytest.approx(0.5 * (1 + math.erf(1 / math.sqrt(2))), rel=1e-15)
    assert M.gelu(np.array([-30.0]))[0] == pytest.approx(0.0, abs=1e-12)


def test_mlp_gradients_central_differences():
    p = M.init_params(out_dim=12, hidden=7, seed=1)
    for k in ("b1", "b2", "b3"):
        p[k] = np.random.default_rng(2).standard_normal(p[k].shape) * 0.1
    g = np.array([0.1, 0.5, 0.9])
    tgt = np.random.default_rng(3).standard_normal((3, 12))
    _, gr = M.loss_and_grads(p, g, tgt, bf16_weights=False)
    h = 1e-6
    for k in M.PARAMS:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 5)):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = M.loss_and_grads(p, g, tgt, bf16_weights=False)
            flat[idx] = old - h
            lm, _ = M.loss_and_grads(p, g, tgt, bf16_weights=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert gr[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_adam_first_step_is_lr_times_sign():
    p = {k: np.ones(3) for k in M.PARAMS}
    gr = {k: np.array([2.0, -3.0, 0.5]) for k in M.PARAMS}
    st = {}
    M.adam_step(p, gr, st, lr=0.01)
    np.testing.assert_allclose(p["W1"], 1.0 - 0.01 * np.sign(gr["W1"]), rtol=1e-6)

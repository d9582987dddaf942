"""Vector and block Lanczos in plain FP64 numpy (oracle; test infrastructure only).

Follows Sec. II of Zbikowski & Johnson, "Bootstrapped Block Lanczos for
large-dimension eigenvalue problems" (arXiv 2210.15763):

  vector_lanczos   Algorithm 1 (steps 1-6) with full reorthogonalisation of
                   each new vector against all previous ones (Sec. II.A).
  block_lanczos_thick  the same iteration with thick restart (the remedy
                   Sec. II.A names for the storage of all vectors): when the
                   basis is full, keep the `keep` lowest Ritz vectors and the
                   newest block, and go on.  The projected matrix is then an
                   arrowhead: the kept Ritz values on the diagonal, coupled
                   to the newest block only (by B_J times the last block row
                   of the kept Ritz vectors' coordinates).
  block_lanczos    Eqs. 4-12 (Sec. II.B): W = H V_n; A_n; subtraction;
                   full reorthogonalisation; normalisation into V_{n+1} and
                   B_n, either by the paper's spectral decomposition of the
                   overlap matrix (Eqs. 9-11) or by CholQR2; block
                   tridiagonal T (Eq. 12) solved by LAPACK (numpy.linalg.eigh).

Readings of garbled or silent passages (each also listed in the design notes):
  * Eq. 7 is printed as W^T W = A_n; it is read as A_n = V_n^T W_n = V_n^T H V_n,
    symmetrised as (A + A^T)/2.
  * Eq. 8 omits the previous block; the subtraction used is
    W' = W - V_n A_n - V_{n-1} B_{n-1}^T (the term implied by Eq. 6).
  * Eq. 10 is printed as B_n = sqrt(Lambda U^T); it is read as
    B_n = Lambda^{1/2} U^T, so that B_n^T B_n = O and V_{n+1} B_n = W'.
  * Eq. 12: block (i+1, i) of T holds B_i and block (i, i+1) holds B_i^T;
    the last off-diagonal index is k-1 (not k).
  * Full reorthogonalisation (Sec. II.A) is two passes of classical block
    Gram-Schmidt against all stored blocks ("twice is enough").
  * Convergence: ||B_n s_i[last b]||_2 <= tol * ||H||_inf for all of the
    nev lowest Ritz pairs at once (default), or the paper's rms change of
    the nev lowest Ritz values below a threshold (Sec. III.A).
  * Breakdown / near-singular overlap ("easy to locate and remove", Sec. II.B):
    a column whose orthogonal part has norm below defl_tol * ||H||_inf is
    replaced by a splitmix64 uniform vector orthogonalised against the basis,
    and the matching part of B_n is set to zero.  In the spectral normaliser
    an eigenvalue of the overlap O also counts as near-singular at or below
    1e-14 times O's largest (the eigensolve of O resolves no finer).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import rng as _rng
from .spmm import norm_inf, spmm

DEFLATION_SEED_XOR = 0x5DEECE66D
# eigenvalues of the overlap matrix O (Eq. 9) below this fraction of its
# largest are numerically zero (about 50 times the FP64 machine epsilon)
NEAR_SINGULAR_REL = 1e-14


# --------------------------------------------------------------------------
# small dense helpers (textbook, Golub & Van Loan)
# --------------------------------------------------------------------------
def cholesky_deflate(G: np.ndarray, thresh2: float):
    """Upper Cholesky factor R of G = R^T R, column by column.

    A pivot d_i <= thresh2 marks column i as numerically dependent: row i of
    R is left zero and i is returned in the deflated list."""
    b = G.shape[0]
    R = np.zeros((b, b))
    deflated = []
    for i in range(b):
        d = G[i, i] - np.dot(R[:i, i], R[:i, i])
        if not d > thresh2:
            deflated.append(i)
            continue
        R[i, i] = np.sqrt(d)
        for k in range(i + 1, b):
            R[i, k] = (G[i, k] - np.dot(R[:i, i], R[:i, k])) / R[i, i]
    return R, deflated


def solve_upper_right(W: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Returns W R^{-1} for upper-triangular nonsingular R (back substitution per row)."""
    b = R.shape[0]
    Q = np.zeros_like(W)
    for c in range(b):
        acc = W[:, c] - Q[:, :c] @ R[:c, c]
        Q[:, c] = acc / R[c, c]
    return Q


def cgs_pass(W: np.ndarray, basis: np.ndarray) -> np.ndarray:
    """One classical block Gram-Schmidt pass: W - Q (Q^T W)."""
    if basis is None or basis.shape[1] == 0:
        return W
    return W - basis @ (basis.T @ W)


def deflation_vector(seed: int, j: int, i: int, n: int) -> np.ndarray:
    """Uniform(-1,1) replacement for column i of block j (splitmix64 counters)."""
    k = np.arange(n, dtype=np.uint64) + np.uint64((j * 64 + i) * n)
    return 2.0 * _rng.uniform01(seed ^ DEFLATION_SEED_XOR, k) - 1.0


def cholqr2(W: np.ndarray, thresh2: float, basis: np.ndarray | None = None, replace=None):
    """CholQR2 with deflation: returns (Q, B, deflated) with W = Q B up to deflated parts.

    G1 = W^T W, R1 = chol(G1), Q1 = W R1^{-1}; G2 = Q1^T Q1, R2 = chol(G2),
    Q = Q1 R2^{-1}; B = R2 R1.  If column i of W is numerically dependent it is
    replaced by replace(i), orthogonalised twice against `basis`, and
    B = triu(Q^T W) so that only the dependent part of W is dropped."""
    W_in = W.copy()
    W = W.copy()
    G1 = W.T @ W
    R1, defl = cholesky_deflate(G1, thresh2)
    if defl:
        for i in defl:
            r = replace(i)[:, None]
            r = cgs_pass(cgs_pass(r, basis), basis)
            W[:, i] = r[:, 0]
        G1 = W.T @ W
        R1, defl2 = cholesky_deflate(G1, 0.0)
        if defl2:
            raise FloatingPointError("deflation replacement vectors are dependent")
    Q1 = solve_upper_right(W, R1)
    R2, d2 = cholesky_deflate(Q1.T @ Q1, 0.0)
    if d2:
        raise FloatingPointError("CholQR2 second pass lost positive definiteness")
    Q = solve_upper_right(Q1, R2)
    if defl:
        B = np.triu(Q.T @ W_in)
    else:
        B = R2 @ R1
    return Q, B, defl


def spectral_normalise(W: np.ndarray, thresh2: float, basis: np.ndarray | None = None, replace=None):
    """The paper's normaliser (Eqs. 9-11): O = W'^T W' = U Lambda U^T,
    B = Lambda^{1/2} U^T, V_{n+1} = W' U Lambda^{-1/2}; near-singular
    eigenvalues of O (Sec. II.B) are removed: their rows of B are zero and
    their columns of V_{n+1} are replaced by vectors orthogonal to everything
    else.  An eigenvalue counts as near-singular at or below thresh2, or at or
    below NEAR_SINGULAR_REL * lambda_max: the eigenvalues of O are only known
    to about machine epsilon times lambda_max, so a direction that W' lacks
    exactly can come out of the eigensolve anywhere below that level."""
    O = W.T @ W                                   # Eq. 9
    lam, U = np.linalg.eigh(O)
    b = W.shape[1]
    B = np.zeros((b, b))
    V = np.zeros_like(W)
    removed = []
    cut = max(thresh2, NEAR_SINGULAR_REL * max(float(lam[-1]), 0.0))
    for c in range(b):
        if lam[c] > cut:
            B[c, :] = np.sqrt(lam[c]) * U[:, c]       # Eq. 10 read as Lambda^{1/2} U^T
            V[:, c] = (W @ U[:, c]) / np.sqrt(lam[c])  # Eq. 11
        else:
            removed.append(c)
    for c in removed:
        kept = np.array([k for k in range(b) if k not in removed] + [k for k in removed if k < c], dtype=int)
        others = V[:, kept] if kept.size else None
        full = others if basis is None else (basis if others is None else np.hstack([basis, others]))
        r = replace(c)[:, None]
        r = cgs_pass(cgs_pass(r, full), full)
        V[:, c] = r[:, 0] / np.linalg.norm(r)
    return V, B, removed


def block_tridiagonal(A: list, B: list) -> np.ndarray:
    """Eq. 12: A_i on the diagonal, B_i in block (i+1, i), B_i^T in block (i, i+1)."""
    J = len(A)
    b = A[0].shape[0]
    T = np.zeros((J * b, J * b))
    for i in range(J):
        T[i * b:(i + 1) * b, i * b:(i + 1) * b] = A[i]
    for i in range(J - 1):
        T[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] = B[i]
        T[i * b:(i + 1) * b, (i + 1) * b:(i + 2) * b] = B[i].T
    return T


def sign_normalise(X: np.ndarray) -> np.ndarray:
    """Flips each column so that its first largest-magnitude entry is positive."""
    X = X.copy()
    for c in range(X.shape[1]):
        k = int(np.argmax(np.abs(X[:, c])))
        if X[k, c] < 0:
            X[:, c] = -X[:, c]
    return X


@dataclasses.dataclass
class LanczosResult:
    evals: np.ndarray
    evecs: np.ndarray
    resid: np.ndarray
    resid_est: np.ndarray
    iters: int
    converged: bool
    theta_history: list
    T: np.ndarray
    A: list
    B: list
    V: np.ndarray | None = None
    deflations: int = 0


# --------------------------------------------------------------------------
# Algorithm 1 (vector Lanczos) with full reorthogonalisation
# --------------------------------------------------------------------------
def vector_lanczos(H, v1: np.ndarray, nev: int, tol: float, max_iter: int, reorth_passes: int = 2,
                   keep_basis: bool = False) -> LanczosResult:
    """Algorithm 1, steps 1-6, plus full reorthogonalisation (Sec. II.A)."""
    nrm = norm_inf(H)
    v = np.asarray(v1, dtype=np.float64).reshape(-1)
    v = v / np.linalg.norm(v)
    Vs = [v]
    alpha, beta = [], []
    hist = []
    for i in range(max_iter):
        w = spmm(H, Vs[i][:, None])[:, 0]            # step 1
        a = float(Vs[i] @ w)                          # step 2
        w = w - a * Vs[i]                             # step 3
        if i > 0:
            w = w - beta[i - 1] * Vs[i - 1]           # step 4
        basis = np.stack(Vs, axis=1)
        for _ in range(reorth_passes):                # full reorthogonalisation
            w = w - basis @ (basis.T @ w)
        bnext = float(np.sqrt(w @ w))                 # step 5
        alpha.append(a)
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        theta, S = np.linalg.eigh(T)
        hist.append(theta.copy())
        k = min(nev, len(alpha))
        est = np.abs(bnext * S[-1, :k])
        done = k == nev and np.all(est <= tol * nrm)
        if done or i == max_iter - 1 or bnext == 0.0:
            X = basis @ S[:, :k]
            X = sign_normalise(X)
            R = spmm(H, X) - X * theta[:k]
            return LanczosResult(theta[:k], X, np.linalg.norm(R, axis=0), est, i + 1, bool(done), hist, T,
                                 [np.array([[x]]) for x in alpha], [np.array([[x]]) for x in beta],
                                 basis if keep_basis else None)
        beta.append(bnext)
        Vs.append(w / bnext)                          # step 6
    raise AssertionError("unreachable")


# --------------------------------------------------------------------------
# Block Lanczos (Eqs. 4-12)
# --------------------------------------------------------------------------
def block_lanczos(H, nev: int, b: int, pivot: np.ndarray, tol: float = 1e-8, max_vectors: int = 2000,
                  normaliser: str = "cholqr2", criterion: str = "residual", rms_tol: float = 1e-6,
                  reorth_passes: int = 2, defl_tol: float = 1e-10, seed: int = 0,
                  keep_basis: bool = False) -> LanczosResult:
    """Block Lanczos from the pivot block (n x b) for the nev lowest eigenpairs.

    Per block iteration n (Sec. II.B):
      W = H V_n                                   (Eq. 4)
      A_n = sym(V_n^T W)                          (Eq. 7, read as V^T W)
      W' = W - V_n A_n - V_{n-1} B_{n-1}^T        (Eq. 8 with the Eq. 6 term)
      W' -= Q (Q^T W'), twice, Q = [V_1..V_n]     (full reorthogonalisation)
      V_{n+1}, B_n from W'                        (Eqs. 9-11 or CholQR2)
      T_n (Eq. 12) -> theta, S by LAPACK; residual estimates ||B_n S[last b, i]||.
    """
    n = pivot.shape[0]
    nrm = norm_inf(H)
    thresh2 = (defl_tol * nrm) ** 2
    norm_fn = {"cholqr2": cholqr2, "spectral": spectral_normalise}[normaliser]
    J_max = max(1, max_vectors // b)
    # orthonormalise the pivot block with the same normaliser
    P = np.asarray(pivot, dtype=np.float64)
    pthresh = (1e-10 * max(1e-300, float(np.max(np.linalg.norm(P, axis=0))))) ** 2
    V1, _, d0 = norm_fn(P, pthresh, None, lambda i: deflation_vector(seed, 0, i, n))
    Vs = [V1]
    A, B = [], []
    hist = []
    ndefl = len(d0)
    prev_theta = None
    for j in range(J_max):
        W = spmm(H, Vs[j])                                     # Eq. 4
        Aj = Vs[j].T @ W                                       # Eq. 7 (read)
        Aj = 0.5 * (Aj + Aj.T)
        W = W - Vs[j] @ Aj                                     # Eq. 8
        if j > 0:
            W = W - Vs[j - 1] @ B[j - 1].T                     # Eq. 6 term (reading of Eq. 8)
        basis = np.hstack(Vs)
        for _ in range(reorth_passes):                         # full reorthogonalisation
            W = cgs_pass(W, basis)
        Vn, Bj, d = norm_fn(W, thresh2, basis, lambda i: deflation_vector(seed, j + 1, i, n))
        ndefl += len(d)
        A.append(Aj)
        T = block_tridiagonal(A, B)                            # Eq. 12
        theta, S = np.linalg.eigh(T)                           # "conventional Lapack routines"
        hist.append(theta.copy())
        m = T.shape[0]
        k = min(nev, m)
        est = np.linalg.norm(Bj @ S[m - b:, :k], axis=0)
        if criterion == "residual":
            done = k == nev and bool(np.all(est <= tol * nrm))
        else:
            done = (k == nev and prev_theta is not None and len(prev_theta) >= nev and
                    float(np.sqrt(np.mean((theta[:nev] - prev_theta[:nev]) ** 2))) < rms_tol)
        prev_theta = theta
        if done or j == J_max - 1:
            X = sign_normalise(basis @ S[:, :k])
            R = spmm(H, X) - X * theta[:k]
            return LanczosResult(theta[:k], X, np.linalg.norm(R, axis=0), est, j + 1, bool(done), hist, T,
                                 A, B, basis if keep_basis else None, ndefl)
        Vs.append(Vn)
        B.append(Bj)
    raise AssertionError("unreachable")


# --------------------------------------------------------------------------
# Block Lanczos with thick restart (Sec. II.A names thick restart as the
# remedy for storing every Lanczos vector)
# --------------------------------------------------------------------------
def restarted_projection(theta_kept: np.ndarray, C: np.ndarray, A: list, B: list) -> np.ndarray:
    """The projected matrix Q^T H Q of a restarted basis Q = [X, V_0, V_1, ...]:
    diag(theta_kept) for the kept Ritz vectors X, coupled to the first new
    block V_0 by C (b x keep, block (V_0, X)); then Eq. 12 for the new blocks."""
    k = theta_kept.size
    J = len(A)
    b = A[0].shape[0]
    T = np.zeros((k + J * b, k + J * b))
    T[:k, :k] = np.diag(theta_kept)
    T[k:k + b, :k] = C
    T[:k, k:k + b] = C.T
    T[k:, k:] = block_tridiagonal(A, B)
    return T


def block_lanczos_thick(H, nev: int, b: int, pivot: np.ndarray, tol: float = 1e-8, max_vectors: int = 2000,
                        keep: int = 0, max_blocks: int = 100000, normaliser: str = "cholqr2",
                        reorth_passes: int = 2, defl_tol: float = 1e-10, seed: int = 0,
                        keep_basis: bool = False) -> LanczosResult:
    """Block Lanczos for the nev lowest eigenpairs with thick restart.

    The block step is block_lanczos's (Eqs. 4-12, both Gram-Schmidt passes
    against every stored vector).  When the stored vectors (kept Ritz vectors
    plus blocks) could not take one more block, the restart keeps
    X = Q S[:, :keep] (the keep lowest Ritz vectors), their Ritz values theta
    and the newest block V_{J+1}: since H Q = Q T + V_{J+1} B_J E_J^T, the
    new basis [X, V_{J+1}] has the projection
        [[diag(theta), C^T], [C, A']],   C = B_J E_J^T S[:, :keep],
    and the next block's subtraction (Eq. 8) includes X C^T.  `iters`
    counts every block (SpMM) over all restarts; the run stops after
    max_blocks blocks.  keep = 0: no restart (as block_lanczos)."""
    n = pivot.shape[0]
    nrm = norm_inf(H)
    thresh2 = (defl_tol * nrm) ** 2
    norm_fn = {"cholqr2": cholqr2, "spectral": spectral_normalise}[normaliser]
    if keep and (keep < nev or keep + 2 * b > max_vectors):
        raise ValueError("thick restart needs nev <= keep and keep + 2b <= max_vectors")
    P = np.asarray(pivot, dtype=np.float64)
    pthresh = (1e-10 * max(1e-300, float(np.max(np.linalg.norm(P, axis=0))))) ** 2
    V1, _, d0 = norm_fn(P, pthresh, None, lambda i: deflation_vector(seed, 0, i, n))
    X = np.zeros((n, 0))
    theta_kept = np.zeros(0)
    C = np.zeros((b, 0))
    Vs = [V1]
    A, B = [], []
    hist = []
    ndefl = len(d0)
    restarts = 0
    for blocks in range(1, max_blocks + 1):
        j = len(Vs) - 1
        W = spmm(H, Vs[j])                                     # Eq. 4
        Aj = Vs[j].T @ W                                       # Eq. 7 (read)
        Aj = 0.5 * (Aj + Aj.T)
        W = W - Vs[j] @ Aj                                     # Eq. 8
        if j > 0:
            W = W - Vs[j - 1] @ B[j - 1].T
        elif X.shape[1]:
            W = W - X @ C.T                                    # the restart coupling
        basis = np.hstack([X] + Vs)
        for _ in range(reorth_passes):                         # full reorthogonalisation
            W = cgs_pass(W, basis)
        Vn, Bj, d = norm_fn(W, thresh2, basis, lambda i: deflation_vector(seed, blocks, i, n))
        ndefl += len(d)
        A.append(Aj)
        T = restarted_projection(theta_kept, C, A, B) if X.shape[1] else block_tridiagonal(A, B)
        theta, S = np.linalg.eigh(T)
        hist.append(theta.copy())
        m = T.shape[0]
        k = min(nev, m)
        est = np.linalg.norm(Bj @ S[m - b:, :k], axis=0)
        done = k == nev and bool(np.all(est <= tol * nrm))
        full = X.shape[1] + (j + 2) * b > max_vectors
        if done or blocks == max_blocks or (full and not keep):
            Xr = sign_normalise(basis @ S[:, :k])
            R = spmm(H, Xr) - Xr * theta[:k]
            res = LanczosResult(theta[:k], Xr, np.linalg.norm(R, axis=0), est, blocks, bool(done), hist, T,
                                A, B, basis if keep_basis else None, ndefl)
            res.restarts = restarts
            return res
        if full:                                               # thick restart
            Sk = S[:, :keep]
            X = basis @ Sk
            theta_kept = theta[:keep].copy()
            C = Bj @ Sk[m - b:, :]
            Vs, A, B = [Vn], [], []
            restarts += 1
        else:
            Vs.append(Vn)
            B.append(Bj)
    raise AssertionError("unreachable")

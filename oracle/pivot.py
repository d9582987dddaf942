"""Pivot blocks (oracle; test infrastructure only).

random_pivot     i.i.d. N(0,1) block ("randomly constructed pivot", Sec. III),
                 from the splitmix64 counter generator.
pivot_overlap    Sec. II.B / III.A: the share of each eigenvector inside the
                 span of the pivot, ||Q^T x|| with Q an orthonormal basis of
                 span(P) (Householder QR).
bootstrap_pivot  Sec. II.B (bootstrapping) and Sec. III: approximate lowest
                 eigenvectors computed in a truncated space, projected into
                 the full space.  The truncated space is the set S of the
                 `trunc_dim` basis states with the lowest diagonal entries
                 H_ii (ties: lower index first), the analogue of the paper's
                 W / N_max truncations for matrices without a physics basis;
                 "projection" embeds the truncated eigenvectors by index, with
                 zeros outside S.  The truncated problem H[S, S] is solved by
                 a dense LAPACK eigensolver.  If b exceeds |S| the remaining
                 columns are random (then the block is orthonormalised by the
                 solver).
"""
import numpy as np

from . import rng as _rng
from .spmm import as_scipy


def random_pivot(n: int, b: int, seed: int) -> np.ndarray:
    return _rng.normal_block(seed, n, b)


def truncated_set(diag: np.ndarray, trunc_dim: int) -> np.ndarray:
    """Indices of the trunc_dim smallest diagonal entries, ties by lower index, returned ascending."""
    order = np.lexsort((np.arange(diag.size), diag))
    return np.sort(order[:trunc_dim])


def bootstrap_pivot(H, trunc_dim: int, b: int, seed: int = 0):
    """Returns (pivot n x b, S, truncated eigenvalues)."""
    Hs = as_scipy(H).tocsr()
    n = Hs.shape[0]
    trunc_dim = int(min(trunc_dim, n))
    S = truncated_set(Hs.diagonal(), trunc_dim)
    Hss = Hs[S][:, S].toarray()
    theta, Y = np.linalg.eigh(Hss)
    k = min(b, trunc_dim)
    P = np.zeros((n, b))
    P[S, :k] = Y[:, :k]
    if k < b:
        P[:, k:] = _rng.normal_block(seed, n, b - k)
    return P, S, theta[:k]


def pivot_overlap(P: np.ndarray, X: np.ndarray, rank_tol: float = 1e-10) -> np.ndarray:
    """||Q^T x_i||_2 for each column of X, Q an orthonormal basis of span(P)
    (Householder QR; directions with |R_ii| below rank_tol * max |R_jj| are
    dropped)."""
    Q, R = np.linalg.qr(np.asarray(P, dtype=np.float64))
    d = np.abs(np.diag(R))
    Q = Q[:, d > rank_tol * d.max()] if d.size and d.max() > 0 else Q[:, :0]
    return np.linalg.norm(Q.T @ np.asarray(X, dtype=np.float64), axis=0)

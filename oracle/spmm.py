"""Sparse matrix times dense block, W = H V (Sec. II.B, Eq. 3: w_{a,i} = sum_j H_ij v_{a,j}).

Blocks are n x b with the block index a contiguous for each row (the paper's
row-wise storage of W^T, Eq. 5).  `spmm` uses scipy's CSR product as the
library primitive; `spmm_loops` is the definition written out as loops for
tiny inputs (it pins `spmm`).
"""
import numpy as np


def as_scipy(H):
    """Accepts a scipy sparse matrix or anything with .to_scipy() (synth.CSR)."""
    return H.to_scipy() if hasattr(H, "to_scipy") else H


def spmm(H, V: np.ndarray) -> np.ndarray:
    """W = H V in FP64 (Eq. 3)."""
    return np.asarray(as_scipy(H) @ np.asarray(V, dtype=np.float64))


def spmm_loops(row_ptr, col, val, V: np.ndarray) -> np.ndarray:
    """Eq. 3 as written: loop over stored elements (i, j, H_ij), inner loop over a."""
    n, b = V.shape
    W = np.zeros((n, b))
    for i in range(n):
        for e in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            j = int(col[e])
            h = float(val[e])
            for a in range(b):
                W[i, a] += h * V[j, a]
    return W


def spmm_rows(H, V: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Selected rows of W = H V, each computed on its own (sampled checks at full size)."""
    Hs = as_scipy(H)
    return np.asarray(Hs[rows] @ V)


def norm_inf(H) -> float:
    """||H||_inf = max absolute row sum (the scale of the residual test)."""
    Hs = as_scipy(H)
    return float(np.abs(Hs).sum(axis=1).max()) if Hs.shape[0] else 0.0

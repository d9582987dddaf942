"""Helpers shared by the GPU tests (no solver arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA GPU")
    import paper_2210_15763_gb300 as bbl
    return torch, bbl


def to_dev(torch, x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def abs_bound(A, V):
    """|H| |V| entrywise (the scale of the rounding error of each W entry)."""
    import scipy.sparse as sp
    Hs = A.to_scipy()
    return np.asarray(abs(Hs) @ np.abs(V))


def principal_angle_sin(X, Y):
    """sin of the largest principal angle between span(X) and span(Y) (orthonormal columns)."""
    s = np.linalg.svd(X.T @ Y, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - min(s) ** 2)))

"""SpMM schedule autotuner.

For a matrix (or a stacked batch of matrices) it times the library's SpMM
under each candidate schedule -- CSR with 2..32 lanes per row, SELL-C-sigma
(C = 32 rows per slice) with several sorting windows sigma -- with CUDA
events, and keeps the fastest.  Results are cached in a JSON table keyed by
the matrix class (storage precision, block size, dimension and
nonzeros-per-row buckets), so later matrices of the same class skip the
timing.  The table lives at $BBL_AUTOTUNE_CACHE or
~/.cache/bbl/spmm_autotune.json.
"""
from __future__ import annotations

import json
import math
import os

CSR_LANES = (2, 4, 8, 16, 32)
SELL_SIGMAS = (32, 256, 1024)


def cache_path() -> str:
    return os.environ.get("BBL_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bbl", "spmm_autotune.json"))


def matrix_class(n: int, nnz: int, b: int, storage: str) -> str:
    """Bucket key: storage, b, log2 of n, log2 of nonzeros per row."""
    per_row = nnz / max(n, 1)
    return f"{storage}/b{b}/n2^{int(math.log2(max(n, 1)))}/r2^{int(math.log2(max(per_row, 1.0)))}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(table: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def time_spmm(A, b: int, lanes=None, reps: int = 5) -> float:
    """Average milliseconds of one SpMM launch (CUDA events, after a warm-up)."""
    import torch
    from . import spmm
    V = torch.randn(A.n, b, device="cuda", dtype=A.dtype)
    W = torch.empty_like(V)
    spmm(A, V, W, lanes_per_row=lanes)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        spmm(A, V, W, lanes_per_row=lanes)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(csr, b: int, storage: str = "fp32", reps: int = 5, use_cache: bool = True, sell: bool = True) -> dict:
    """Best SpMM schedule for `csr` (host CSR) at block size b.

    Returns {"fmt": "csr"|"sell", "lanes": L, "sigma": S, "ms": t, "class": key, "timings": [...]}."""
    from . import Matrix
    n, nnz = int(csr.n), int(csr.row_ptr[-1])
    key = matrix_class(n, nnz, b, storage)
    table = _load() if use_cache else {}
    if use_cache and key in table:
        return dict(table[key], cached=True)
    timings = []
    A = Matrix(csr, storage=storage, fmt="csr")
    for L in CSR_LANES:
        timings.append({"fmt": "csr", "lanes": L, "sigma": 0, "ms": time_spmm(A, b, lanes=L, reps=reps)})
    A.close()
    if sell:
        for s in SELL_SIGMAS:
            As = Matrix(csr, storage=storage, fmt="sell", sell_sigma=s)
            timings.append({"fmt": "sell", "lanes": 0, "sigma": s, "ms": time_spmm(As, b, reps=reps)})
            As.close()
    best = min(timings, key=lambda t: t["ms"])
    out = dict(best, **{"class": key, "timings": timings})
    if use_cache:
        table[key] = out
        _store(table)
    return dict(out, cached=False)

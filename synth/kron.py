"""Seeded synthetic inputs shared by the oracle and the GPU path.

The paper's matrices are nuclear configuration-interaction Hamiltonians
(Sec. III, Appendix A) that are not available here.  They are replaced by
seeded random matrices with the same "proton x neutron" factorised structure
the paper exploits for on-the-fly reconstruction (Sec. III, Appendix A):

    H = Hp (x) I + I (x) Hn + sum_{k=1..K} Cp_k (x) Cn_k

Hp, Hn are symmetric with about ``d_off`` off-diagonal N(0,1) entries per row
and a diagonal of sorted U(0,20) draws; every coupling factor Cp_k, Cn_k is
symmetric with about ``c`` nonzeros per row (one diagonal entry plus mirrored
off-diagonals), values N(0, 0.5^2).  All factor entries are rounded to FP32
and every assembled entry of H is rounded to FP32 once, so that the FP64 and
the FP32-storage solvers see exactly the same matrix.

This module holds no eigensolver arithmetic: only random draws, the
Kronecker expansion (synth/kron_csr.c) and textbook test matrices.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kron_csr.c")
_LIB = os.path.join(_HERE, "_kron_csr.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the Kronecker assembler with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            f = lib.kron_assemble
            f.restype = ctypes.c_int64
            f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 9 + [ctypes.c_int]
            _lib = lib
    return _lib


# --------------------------------------------------------------------------
# CSR container
# --------------------------------------------------------------------------
@dataclasses.dataclass
class CSR:
    """Square sparse matrix in CSR form: int64 row_ptr, int32 col, FP64 or FP32 val."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.astype(np.float64), self.col, self.row_ptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col), self.val.astype(np.float64))
        return d

    def diagonal(self) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d = np.zeros(self.n)
        m = rows == self.col
        d[rows[m]] = self.val[m]
        return d


def csr_from_scipy(a) -> CSR:
    a = a.tocsr()
    a.sort_indices()
    a.sum_duplicates()
    return CSR(a.shape[0], a.indptr.astype(np.int64), a.indices.astype(np.int32), a.data.astype(np.float64))


def csr_from_dense(d: np.ndarray) -> CSR:
    import scipy.sparse as sp
    return csr_from_scipy(sp.csr_matrix(d))


# --------------------------------------------------------------------------
# Factor matrices
# --------------------------------------------------------------------------
def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _sym_factor(rng, N: int, n_pairs: int, off_sigma: float, diag: np.ndarray):
    """Symmetric sparse N x N factor: `n_pairs` random (i<j) pairs mirrored, plus `diag`."""
    i = rng.integers(0, N, size=n_pairs)
    j = rng.integers(0, N, size=n_pairs)
    v = _f32(rng.standard_normal(n_pairs) * off_sigma)
    keep = i != j
    i, j, v = i[keep], j[keep], v[keep]
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    key = lo.astype(np.int64) * N + hi
    _, first = np.unique(key, return_index=True)
    lo, hi, v = lo[first], hi[first], v[first]
    rows = np.concatenate([lo, hi, np.arange(N)])
    cols = np.concatenate([hi, lo, np.arange(N)])
    vals = np.concatenate([v, v, _f32(diag)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    ptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(ptr, rows + 1, 1)
    return CSR(N, np.cumsum(ptr), cols.astype(np.int32), vals)


def h_factor(rng, N: int, d_off: float) -> CSR:
    """Hp / Hn: ~d_off off-diagonal N(0,1) entries per row, diagonal sorted U(0,20)."""
    diag = np.sort(rng.uniform(0.0, 20.0, size=N))
    return _sym_factor(rng, N, int(round(N * d_off / 2)), 1.0, diag)


def c_factor(rng, N: int, c: float, sigma: float = 0.5) -> CSR:
    """Cp_k / Cn_k: ~c nonzeros per row (diagonal + mirrored off-diagonals), N(0, sigma^2)."""
    diag = rng.standard_normal(N) * sigma
    return _sym_factor(rng, N, int(round(N * max(c - 1.0, 0.0) / 2)), sigma, diag)


@dataclasses.dataclass
class KronFactors:
    Hp: CSR
    Hn: CSR
    Cp: list
    Cn: list

    @property
    def n(self) -> int:
        return self.Hp.n * self.Hn.n


def kron_factors(nP: int, nN: int, K: int, c: float, seed: int, d_off: float = 10.0,
                 sigma_c: float = 0.5) -> KronFactors:
    rng = np.random.default_rng(seed)
    Hp = h_factor(rng, nP, d_off)
    Hn = h_factor(rng, nN, d_off)
    Cp, Cn = [], []
    for _ in range(K):
        Cp.append(c_factor(rng, nP, c, sigma_c))
        Cn.append(c_factor(rng, nN, c, sigma_c))
    return KronFactors(Hp, Hn, Cp, Cn)


def assemble(f: KronFactors, fp32_values: bool = False, extra_scale: float | None = None,
             extra: KronFactors | None = None, exact: bool = False) -> CSR:
    """Expands the Kronecker sum into CSR.

    With ``extra`` given, its coupling terms are appended with their Cp values
    multiplied by ``extra_scale`` (used for the family H(g) = H0 + g V).
    ``exact`` keeps every entry as the FP64 sum of its factor products (no
    FP32 rounding): the matrix that an operator applying the factors
    themselves applies (FP64 values only).
    """
    if exact and fp32_values:
        raise ValueError("exact entries are FP64 sums of factor products")
    cp, cn = list(f.Cp), list(f.Cn)
    if extra is not None:
        s = 1.0 if extra_scale is None else float(extra_scale)
        for a, b in zip(extra.Cp, extra.Cn):
            cp.append(CSR(a.n, a.row_ptr, a.col, a.val * s))
            cn.append(b)
    facs = [f.Hp, f.Hn]
    for a, b in zip(cp, cn):
        facs += [a, b]
    ptrs = np.concatenate([x.row_ptr for x in facs]).astype(np.int64)
    idxs = np.concatenate([x.col for x in facs]).astype(np.int32)
    vals = np.concatenate([x.val for x in facs]).astype(np.float64)
    offs_ptr = np.cumsum([0] + [x.n + 1 for x in facs[:-1]]).astype(np.int64)
    offs_nz = np.cumsum([0] + [x.nnz for x in facs[:-1]]).astype(np.int64)
    nP, nN, K = f.Hp.n, f.Hn.n, len(cp)
    n = nP * nN
    lib = _load()
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    r32 = 0 if exact else 1
    nnz = lib.kron_assemble(nP, nN, K, p(ptrs), p(idxs), p(vals), p(offs_ptr), p(offs_nz),
                            p(row_ptr), None, None, None, r32)
    if nnz < 0:
        raise MemoryError("kron_assemble: out of memory (pass 1)")
    col = np.empty(nnz, dtype=np.int32)
    if fp32_values:
        val = np.empty(nnz, dtype=np.float32)
        r = lib.kron_assemble(nP, nN, K, p(ptrs), p(idxs), p(vals), p(offs_ptr), p(offs_nz),
                              p(row_ptr), p(col), None, p(val), r32)
    else:
        val = np.empty(nnz, dtype=np.float64)
        r = lib.kron_assemble(nP, nN, K, p(ptrs), p(idxs), p(vals), p(offs_ptr), p(offs_nz),
                              p(row_ptr), p(col), p(val), None, r32)
    if r < 0:
        raise MemoryError("kron_assemble: out of memory (pass 2)")
    return CSR(n, row_ptr, col, val)


# --------------------------------------------------------------------------
# Named workloads (synthetic stand-ins for the paper's Sec. III matrices)
# --------------------------------------------------------------------------
# The coupling density c is chosen so that the measured nonzeros per row come
# close to the stated totals (~100 for n=2e4, ~300 for n=2e6, ~200 for n=2e7):
# with ~21 entries from Hp(x)I + I(x)Hn, each coupling term adds ~c^2.
KRON_CONFIGS = {
    "kron_n2e4": dict(nP=200, nN=100, K=4, c=4.75, seed=20221028),
    "kron_n2e6": dict(nP=2000, nN=1000, K=12, c=4.8, seed=20221029),
    "kron_n2e7": dict(nP=5000, nN=4000, K=12, c=3.9, seed=20221030),
    "kron_n2e6_c3": dict(nP=2000, nN=1000, K=12, c=3.9, seed=20221030),
    "kron_n1e6_h0": dict(nP=1000, nN=1000, K=12, c=3.9, seed=20221031),
}


def kron_config(name: str, scale: float = 1.0) -> dict:
    """Parameters of a named workload; ``scale`` < 1 shrinks both factors (tests)."""
    cfg = dict(KRON_CONFIGS[name])
    if scale != 1.0:
        cfg["nP"] = max(4, int(round(cfg["nP"] * scale)))
        cfg["nN"] = max(4, int(round(cfg["nN"] * scale)))
    return cfg


def named_factors(name: str, scale: float = 1.0, K: int | None = None) -> KronFactors:
    """The factor matrices of a named workload."""
    cfg = kron_config(name, scale)
    if K is not None:
        cfg["K"] = K
    return kron_factors(cfg["nP"], cfg["nN"], cfg["K"], cfg["c"], cfg["seed"])


def kron_matrix(name: str, scale: float = 1.0, fp32_values: bool = False, K: int | None = None,
                exact: bool = False) -> CSR:
    """A named workload assembled into CSR (entries rounded to FP32 unless
    ``exact``; a name ending in "_exact" asks for the exact entries)."""
    if name.endswith("_exact"):
        name, exact = name[:-len("_exact")], True
    return assemble(named_factors(name, scale, K), fp32_values=fp32_values, exact=exact)


def learned_family(scale: float = 1.0, seed: int = 20221032):
    """H(g) = H0 + g V: H0 is the n=1e6 Kronecker matrix, V six further
    random Kronecker coupling terms with ~3 nonzeros per factor row."""
    cfg = kron_config("kron_n1e6_h0", scale)
    h0 = kron_factors(cfg["nP"], cfg["nN"], cfg["K"], cfg["c"], cfg["seed"])
    rng = np.random.default_rng(seed)
    v = KronFactors(h0.Hp, h0.Hn, [c_factor(rng, cfg["nP"], 3.0) for _ in range(6)],
                    [c_factor(rng, cfg["nN"], 3.0) for _ in range(6)])
    return h0, v


def family_matrix(h0: KronFactors, v: KronFactors, g: float, fp32_values: bool = False) -> CSR:
    return assemble(h0, fp32_values=fp32_values, extra=v, extra_scale=g)


def family_g(seed: int = 20221033, count: int = 64):
    """g ~ U(0,1), seeded; the first 48 are training values, the last 16 held out."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=count)


def batch_matrices(count: int = 256, seed: int = 20221034, n_lo: float = 2e3, n_hi: float = 2e5):
    """Uneven batch: n log-uniform in [n_lo, n_hi], ~50-150 nonzeros per row.

    Returns the list of (nP, nN, K, c, seed) parameter dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        nP = max(8, int(round(np.sqrt(n * 2.0))))
        nN = max(4, int(round(n / nP)))
        target = rng.uniform(50.0, 150.0)
        K = 4
        c = float(np.sqrt(max(target - 21.0, 1.0) / K))
        out.append(dict(nP=nP, nN=nN, K=K, c=c, seed=seed + 1 + i))
    return out


# --------------------------------------------------------------------------
# Textbook matrices with closed-form spectra
# --------------------------------------------------------------------------
def laplacian_1d(n: int) -> CSR:
    """Dirichlet 1-D Laplacian tridiag(-1, 2, -1)."""
    rows, cols, vals = [], [], []
    for i in range(n):
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(-1.0)
        rows.append(i); cols.append(i); vals.append(2.0)
        if i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(-1.0)
    import scipy.sparse as sp
    return csr_from_scipy(sp.csr_matrix((vals, (rows, cols)), shape=(n, n)))


def laplacian_2d(nx: int, ny: int) -> CSR:
    """L_x (x) I + I (x) L_y with Dirichlet 1-D Laplacians."""
    import scipy.sparse as sp
    lx = laplacian_1d(nx).to_scipy()
    ly = laplacian_1d(ny).to_scipy()
    return csr_from_scipy(sp.kron(lx, sp.identity(ny)) + sp.kron(sp.identity(nx), ly))


def random_sparse_symmetric(n: int, per_row: float, seed: int, empty_rows: int = 0,
                            long_row: int = 0) -> CSR:
    """Random symmetric matrix with FP32-exact values; optional empty rows at
    the end and one dense-ish 'long' row (row 0) coupled to `long_row` columns."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    m = n - empty_rows
    pairs = int(round(m * per_row / 2))
    i = rng.integers(0, m, size=pairs)
    j = rng.integers(0, m, size=pairs)
    v = _f32(rng.standard_normal(pairs))
    keep = i != j
    lo, hi, v = np.minimum(i, j)[keep], np.maximum(i, j)[keep], v[keep]
    if long_row > 0 and m > 1:
        jj = rng.choice(np.arange(1, m), size=min(long_row, m - 1), replace=False)
        lo = np.concatenate([lo, np.zeros_like(jj)])
        hi = np.concatenate([hi, jj])
        v = np.concatenate([v, _f32(rng.standard_normal(jj.size))])
    upper = sp.coo_matrix((v, (lo, hi)), shape=(n, n)).tocsr()
    upper.sum_duplicates()
    upper.data = _f32(upper.data)
    d = np.zeros(n)
    d[:m] = _f32(rng.uniform(-5, 5, size=m))
    return csr_from_scipy(upper + upper.T + sp.diags(d))


def gaussian_block(n: int, b: int, seed: int) -> np.ndarray:
    """i.i.d. N(0,1) n x b block (row-major), e.g. a random pivot."""
    return np.random.default_rng(seed).standard_normal((n, b))

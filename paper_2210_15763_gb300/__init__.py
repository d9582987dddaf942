"""GB300-native bootstrapped block Lanczos (Zbikowski & Johnson, arXiv 2210.15763).

Thin Python binding of the C ABI declared in include/bbl.h.  Every step of
the eigensolver runs in the CUDA library libbbl.so; this module only
marshals arguments.  PyTorch provides device memory and streams.  There is
no CPU fallback: the functions raise if the library cannot be loaded or no
GPU is present.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import _lib
from ._lib import BBLError, CSR, FP32, FP64, SELL, Options, Stats

__all__ = ["Matrix", "KronMatrix", "spmm", "spmm_f64", "block_reorth", "cholqr2", "ritz_banded", "ritz_vectors", "pivot_random",
           "pivot_bootstrap", "solve", "SolveResult", "BBLError", "options", "FP32", "FP64", "CSR", "SELL"]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2210_15763_gb300 needs a CUDA GPU (no CPU fallback)")
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(C.c_void_p)
    return C.c_void_p(int(x))


def _dtype_code(t) -> int:
    torch = _torch()
    if t == torch.float64:
        return FP64
    if t == torch.float32:
        return FP32
    raise TypeError(f"unsupported dtype {t}")


def options(**kw) -> Options:
    """bbl_options with defaults from bbl_options_default, overridden by keywords."""
    lib = _lib.load()
    o = Options()
    lib.bbl_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "stream":
            o.stream = _stream(v)
        elif k == "storage" and isinstance(v, str):
            o.storage = FP32 if v == "fp32" else FP64
        else:
            setattr(o, k, v)
    return o


class Matrix:
    """Device copy of a sparse symmetric matrix (bbl_matrix).

    `csr` is anything with n, row_ptr (int64), col (int32) and val (float64 or
    float32) as numpy arrays or torch tensors (host or device).  fmt: "csr",
    "sell" (sell_sigma = sorting window) or "tiled" (sell_sigma = tile size)."""

    def __init__(self, csr, storage: str = "fp64", fmt: str = "csr", sell_sigma: int = 0, keep_fp64: bool = False,
                 check_symmetry: bool = False, stream=None):
        lib = _lib.load()
        self._lib = lib
        rp, col, val = csr.row_ptr, csr.col, csr.val
        if isinstance(rp, np.ndarray):
            rp = np.ascontiguousarray(rp, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            if val.dtype not in (np.float64, np.float32):
                val = val.astype(np.float64)
            val = np.ascontiguousarray(val)
            vdt = FP64 if val.dtype == np.float64 else FP32
        else:
            vdt = _dtype_code(val.dtype)
        self._keep = (rp, col, val)  # keep the arrays alive during the call
        h = C.c_void_p()
        st = lib.bbl_matrix_create(int(csr.n), int(rp[-1]) if isinstance(rp, np.ndarray) else int(rp[-1].item()),
                                   _ptr(rp), _ptr(col), _ptr(val), vdt, FP32 if storage == "fp32" else FP64,
                                   {"sell": SELL, "tiled": _lib.TILED}.get(fmt, CSR), int(sell_sigma), int(keep_fp64),
                                   int(check_symmetry), _stream(stream), C.byref(h))
        self._keep = None
        _lib.check(st)
        self.handle = h
        self.storage = storage
        self.fmt = fmt
        n, nnz, nb, fm, sto, pnz = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int(), C.c_int(), C.c_int64()
        norm = C.c_double()
        _lib.check(lib.bbl_matrix_info(h, C.byref(n), C.byref(nnz), C.byref(norm), C.byref(nb), C.byref(fm),
                                       C.byref(sto), C.byref(pnz)))
        self.n, self.nnz, self.norm_inf, self.device_bytes, self.padded_nnz = n.value, nnz.value, norm.value, nb.value, pnz.value

    @property
    def dtype(self):
        torch = _torch()
        return torch.float32 if self.storage == "fp32" else torch.float64

    def set_spmm_lanes(self, lanes_per_row: int):
        _lib.check(self._lib.bbl_matrix_set_spmm_lanes(self.handle, int(lanes_per_row)))

    def diagonal(self, stream=None):
        torch = _torch()
        d = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _lib.check(self._lib.bbl_matrix_diagonal(self.handle, _ptr(d), _stream(stream)))
        return d

    def close(self):
        if getattr(self, "handle", None):
            self._lib.bbl_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_kron_factors(factors):
    """Layout conversion for bbl_matrix_create_kron: the factors (objects with
    n, row_ptr, col, val) in the order Hp, Hn, Cp_0, Cn_0, ... packed into
    (fptr int32, fcol int32, fval FP64, ptr_off int64, nz_off int64)."""
    facs = [factors.Hp, factors.Hn]
    for a, b in zip(factors.Cp, factors.Cn):
        facs += [a, b]
    ptr_off = np.cumsum([0] + [f.n + 1 for f in facs[:-1]]).astype(np.int64)
    nz_off = np.cumsum([0] + [int(f.row_ptr[-1]) for f in facs[:-1]]).astype(np.int64)
    fptr = np.concatenate([np.asarray(f.row_ptr, dtype=np.int32) for f in facs])
    fcol = np.concatenate([np.asarray(f.col, dtype=np.int32) for f in facs])
    fval = np.concatenate([np.asarray(f.val, dtype=np.float64) for f in facs])
    return fptr, fcol, fval, ptr_off, nz_off


class KronMatrix(Matrix):
    """A matrix kept as its Kronecker factors and applied without storing its
    entries (bbl_matrix_create_kron): H = Hp (x) I + I (x) Hn + sum_k Cp_k (x) Cn_k.
    `factors` has Hp, Hn (CSR-like objects) and the lists Cp, Cn."""

    def __init__(self, factors, storage: str = "fp32", check_symmetry: bool = False, stream=None):
        lib = _lib.load()
        self._lib = lib
        fptr, fcol, fval, ptr_off, nz_off = pack_kron_factors(factors)
        h = C.c_void_p()
        st = lib.bbl_matrix_create_kron(int(factors.Hp.n), int(factors.Hn.n), len(factors.Cp), _ptr(fptr), _ptr(fcol),
                                        _ptr(fval), _ptr(ptr_off), _ptr(nz_off), FP32 if storage == "fp32" else FP64,
                                        int(check_symmetry), _stream(stream), C.byref(h))
        _lib.check(st)
        self.handle = h
        self.storage = storage
        self.fmt = "kron"
        n, nnz, nb, fm, sto, pnz = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int(), C.c_int(), C.c_int64()
        norm = C.c_double()
        _lib.check(lib.bbl_matrix_info(h, C.byref(n), C.byref(nnz), C.byref(norm), C.byref(nb), C.byref(fm),
                                       C.byref(sto), C.byref(pnz)))
        self.n, self.nnz, self.norm_inf, self.device_bytes, self.padded_nnz = n.value, nnz.value, norm.value, nb.value, pnz.value


def spmm(A: Matrix, V, W=None, stream=None, lanes_per_row: int | None = None):
    """W = H V (S1); V, W: CUDA tensors n x b in the matrix storage dtype."""
    torch = _torch()
    b = V.shape[1]
    if W is None:
        W = torch.empty_like(V)
    if lanes_per_row is None:
        _lib.check(A._lib.bbl_spmm(A.handle, b, _ptr(V), _ptr(W), _stream(stream)))
    else:
        _lib.check(A._lib.bbl_spmm_group(A.handle, b, _ptr(V), _ptr(W), int(lanes_per_row), _stream(stream)))
    return W


def spmm_f64(A: Matrix, V, W=None, stream=None):
    """W = H V in FP64 arithmetic (FP64 blocks) whatever the storage."""
    torch = _torch()
    if W is None:
        W = torch.empty_like(V)
    _lib.check(A._lib.bbl_spmm_f64(A.handle, V.shape[1], _ptr(V), _ptr(W), _stream(stream)))
    return W


def block_reorth(basis, W, passes: int = 2, stream=None):
    """Full reorthogonalisation of W (n x b) against basis (nblocks x n x b), in place.
    Returns the FP64 coefficients (passes x nblocks*b x b)."""
    torch = _torch()
    nb, n, b = basis.shape
    coeff = torch.empty((passes, nb * b, b), dtype=torch.float64, device=W.device)
    _lib.check(_lib.load().bbl_block_reorth(n, b, nb, _dtype_code(W.dtype), _ptr(basis), _ptr(W), _ptr(coeff),
                                            passes, _stream(stream)))
    return coeff


def cholqr2(W, defl_abs: float = 0.0, stream=None):
    """CholQR2 in place: W <- Q; returns (B (b x b FP64), number of deflated columns)."""
    torch = _torch()
    n, b = W.shape
    B = torch.empty((b, b), dtype=torch.float64, device=W.device)
    nd = C.c_int()
    _lib.check(_lib.load().bbl_cholqr2(n, b, _dtype_code(W.dtype), _ptr(W), _ptr(B), float(defl_abs), C.byref(nd),
                                       _stream(stream)))
    return B, nd.value


def ritz_banded(Tband, nev: int, stream=None):
    """Lowest nev eigenpairs of the band matrix in lower band storage (m x (p+1))."""
    torch = _torch()
    m, p1 = Tband.shape
    theta = torch.empty(nev, dtype=torch.float64, device=Tband.device)
    S = torch.empty((m, nev), dtype=torch.float64, device=Tband.device)
    _lib.check(_lib.load().bbl_ritz_banded(m, p1 - 1, nev, _ptr(Tband), _ptr(theta), _ptr(S), _stream(stream)))
    return theta, S


def ritz_vectors(basis, S, stream=None):
    """X = Q S (FP64 n x k)."""
    torch = _torch()
    nb, n, b = basis.shape
    k = S.shape[1]
    X = torch.empty((n, k), dtype=torch.float64, device=basis.device)
    _lib.check(_lib.load().bbl_ritz_vectors(n, b, nb, _dtype_code(basis.dtype), _ptr(basis), k, _ptr(S), _ptr(X),
                                            _stream(stream)))
    return X


def pivot_random(n: int, b: int, seed: int, stream=None):
    torch = _torch()
    P = torch.empty((n, b), dtype=torch.float64, device="cuda")
    _lib.check(_lib.load().bbl_pivot_random(n, b, seed, _ptr(P), _stream(stream)))
    return P


def pivot_bootstrap(A: Matrix, trunc_dim: int, b: int, sub_tol: float = 1e-10, seed: int = 0, stream=None):
    torch = _torch()
    P = torch.empty((A.n, b), dtype=torch.float64, device="cuda")
    _lib.check(A._lib.bbl_pivot_bootstrap(A.handle, int(trunc_dim), b, float(sub_tol), seed, _ptr(P), _stream(stream)))
    return P


def block_gram(basis, W, stream=None):
    """C = Q^T W (FP64 m x b) without modifying W."""
    torch = _torch()
    nb, n, b = basis.shape
    C_ = torch.empty((nb * b, b), dtype=torch.float64, device=W.device)
    _lib.check(_lib.load().bbl_block_gram(n, b, nb, _dtype_code(W.dtype), _ptr(basis), _ptr(W), _ptr(C_),
                                          _stream(stream)))
    return C_


def block_gram_f16(basis16, W, stream=None):
    """C ~= Q16^T W (FP64 m x 8) from an FP16 basis copy and FP32 W (b = 8)."""
    torch = _torch()
    nb, n, b = basis16.shape
    if b != 8 or basis16.dtype != torch.float16 or W.dtype != torch.float32:
        raise ValueError("block_gram_f16: FP16 basis of n x 8 blocks and FP32 W")
    C_ = torch.empty((nb * 8, 8), dtype=torch.float64, device=W.device)
    _lib.check(_lib.load().bbl_block_gram_f16(n, nb, _ptr(basis16), _ptr(W), _ptr(C_), _stream(stream)))
    return C_


def block_update_gram(basis, W, C1, stream=None):
    """W -= Q C1 in place, then C2 = Q^T W (FP64 m x 8), in one kernel
    (FP32 basis of n x 8 blocks, at most 128 blocks)."""
    torch = _torch()
    nb, n, b = basis.shape
    if b != 8 or basis.dtype != torch.float32 or W.dtype != torch.float32 or C1.dtype != torch.float64:
        raise ValueError("block_update_gram: FP32 basis of n x 8 blocks, FP32 W, FP64 C1")
    C2 = torch.empty((nb * 8, 8), dtype=torch.float64, device=W.device)
    _lib.check(_lib.load().bbl_block_update_gram(n, nb, _ptr(basis), _ptr(C1.contiguous()), _ptr(W), _ptr(C2),
                                                 _stream(stream)))
    return C2


def block_update_f16old(basis16, basis, W, C, nnew: int = 2, stream=None):
    """W -= Q C in place (FP32, b = 8), the blocks older than the nnew newest
    read from the FP16 copy basis16 (nblocks x n x 8 float16)."""
    torch = _torch()
    nb, n, b = basis.shape
    if b != 8 or basis.dtype != torch.float32 or basis16.dtype != torch.float16 or W.dtype != torch.float32:
        raise ValueError("block_update_f16old: FP32 basis of n x 8 blocks, its FP16 copy, FP32 W")
    _lib.check(_lib.load().bbl_block_update_f16old(n, nb, int(nnew), _ptr(basis16), _ptr(basis),
                                                   _ptr(C.contiguous()), _ptr(W), _stream(stream)))
    return W


def pivot_rr_residual(A: Matrix, P, stream=None):
    """Rayleigh-Ritz values and residual norms of span(P) (the test that chooses a pivot)."""
    b = P.shape[1]
    th = np.zeros(b)
    rs = np.zeros(b)
    if isinstance(P, np.ndarray):
        P = np.ascontiguousarray(P, dtype=np.float64)
    _lib.check(A._lib.bbl_pivot_rr_residual(A.handle, b, _ptr(P), _ptr(th), _ptr(rs), _stream(stream)))
    return th, rs


def pivot_overlap(P, X, stream=None):
    """||orth(P)^T x_i|| for each column x_i of X (host or device FP64)."""
    n, b = P.shape
    k = X.shape[1]
    if isinstance(P, np.ndarray):
        P = np.ascontiguousarray(P, dtype=np.float64)
    if isinstance(X, np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(k)
    _lib.check(_lib.load().bbl_pivot_overlap(n, b, _ptr(P), k, _ptr(X), _ptr(out), _stream(stream)))
    return out


def probe_fma_rate(dtype: str = "fp64", stream=None) -> float:
    """Measured FMA throughput of the GPU in FLOP/s (FP32 or FP64)."""
    out = C.c_double()
    _lib.check(_lib.load().bbl_probe_fma_rate(FP64 if dtype == "fp64" else FP32, C.byref(out), _stream(stream)))
    return out.value


def workspace_bytes() -> int:
    """Bytes of Lanczos bases the library keeps idle for reuse on this device."""
    return int(_lib.load().bbl_workspace_bytes())


def workspace_release():
    """Frees the idle cached bases of the current device."""
    _lib.check(_lib.load().bbl_workspace_release())


class MLP:
    """The learned-pivot network (bbl_mlp): 1 -> hidden -> hidden -> out."""

    def __init__(self, hidden: int, out_dim: int):
        self._lib = _lib.load()
        h = C.c_void_p()
        _lib.check(self._lib.bbl_mlp_create(hidden, out_dim, C.byref(h)))
        self.handle = h
        self.hidden, self.out = hidden, out_dim
        self.nparams = self._lib.bbl_mlp_num_params(h)

    def set_params(self, packed, stream=None):
        packed = np.ascontiguousarray(packed, dtype=np.float32) if isinstance(packed, np.ndarray) else packed
        _lib.check(self._lib.bbl_mlp_set_params(self.handle, _ptr(packed), _stream(stream)))

    def get_params(self, stream=None):
        p = np.zeros(self.nparams, dtype=np.float32)
        g = np.zeros(self.nparams, dtype=np.float32)
        _lib.check(self._lib.bbl_mlp_get_params(self.handle, _ptr(p), _ptr(g), _stream(stream)))
        return p, g

    def forward(self, g, stream=None):
        torch = _torch()
        y = torch.empty((g.shape[0], self.out), dtype=torch.float32, device="cuda")
        _lib.check(self._lib.bbl_mlp_forward(self.handle, g.shape[0], _ptr(g), _ptr(y), _stream(stream)))
        return y

    def loss_grad(self, g, target, stream=None):
        loss = C.c_float()
        _lib.check(self._lib.bbl_mlp_loss_grad(self.handle, g.shape[0], _ptr(g), _ptr(target), C.byref(loss),
                                               _stream(stream)))
        return loss.value

    def adam_step(self, lr: float, stream=None):
        _lib.check(self._lib.bbl_mlp_adam_step(self.handle, float(lr), _stream(stream)))

    def train(self, g, target, epochs: int, lr: float, stream=None):
        hist = np.zeros(max(epochs, 1), dtype=np.float32)
        _lib.check(self._lib.bbl_mlp_train(self.handle, g.shape[0], _ptr(g), _ptr(target), int(epochs), float(lr),
                                           _ptr(hist), _stream(stream)))
        return hist[:epochs]

    def pivot(self, g: float, U, b: int, stream=None):
        """P = U C(g); U: (nblocks, n, bU) FP32 CUDA tensor."""
        torch = _torch()
        nbU, n, bU = U.shape
        P = torch.empty((n, b), dtype=torch.float64, device="cuda")
        _lib.check(self._lib.bbl_pivot_learned(self.handle, float(g), n, bU, nbU, _ptr(U), b, _ptr(P),
                                               _stream(stream)))
        return P

    def close(self):
        if getattr(self, "handle", None):
            self._lib.bbl_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stack_block_diagonal(mats):
    """Stacks square CSR matrices row-wise into one block-diagonal CSR (layout
    conversion for bbl_batch_create): returns (offsets, row_ptr, col, val)."""
    ns = [int(m.n) for m in mats]
    offsets = np.zeros(len(mats) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(ns)
    nnzs = [int(m.row_ptr[-1]) for m in mats]
    nz_off = np.zeros(len(mats) + 1, dtype=np.int64)
    nz_off[1:] = np.cumsum(nnzs)
    row_ptr = np.empty(offsets[-1] + 1, dtype=np.int64)
    col = np.empty(nz_off[-1], dtype=np.int32)
    vdt = np.float32 if all(m.val.dtype == np.float32 for m in mats) else np.float64
    val = np.empty(nz_off[-1], dtype=vdt)
    for s, m in enumerate(mats):
        row_ptr[offsets[s]:offsets[s + 1]] = m.row_ptr[:-1] + nz_off[s]
        col[nz_off[s]:nz_off[s + 1]] = m.col + offsets[s]
        val[nz_off[s]:nz_off[s + 1]] = m.val
    row_ptr[-1] = nz_off[-1]
    return offsets, row_ptr, col, val


class Batch:
    """Many independent problems solved in lock-step (bbl_batch)."""

    def __init__(self, mats, storage: str = "fp32", fmt: str = "csr", sell_sigma: int = 0, stream=None):
        self._lib = _lib.load()
        offsets, rp, col, val = stack_block_diagonal(mats)
        self.count = len(mats)
        self.offsets = offsets
        self.n = int(offsets[-1])
        self.nnz = int(rp[-1])
        self.storage = storage
        h = C.c_void_p()
        _lib.check(self._lib.bbl_batch_create(len(mats), _ptr(offsets), self.nnz, _ptr(rp), _ptr(col), _ptr(val),
                                              FP64 if val.dtype == np.float64 else FP32,
                                              FP32 if storage == "fp32" else FP64, SELL if fmt == "sell" else CSR,
                                              int(sell_sigma), _stream(stream), C.byref(h)))
        self.handle = h

    def set_schedule(self, lanes_per_row: int):
        _lib.check(self._lib.bbl_batch_set_schedule(self.handle, int(lanes_per_row)))

    def solve(self, nev: int, b: int, use_graph: bool = True, **opts):
        o = options(**opts)
        o.storage = FP32 if self.storage == "fp32" else FP64
        if "stream" not in opts:
            o.stream = _stream(None)
        ev = np.zeros((self.count, nev))
        rs = np.zeros((self.count, nev))
        it = np.zeros(self.count, dtype=np.int32)
        stt = np.zeros(self.count, dtype=np.int32)
        st = Stats()
        s = self._lib.bbl_batch_solve(self.handle, nev, b, C.byref(o), int(bool(use_graph)), _ptr(ev), _ptr(rs),
                                      _ptr(it), _ptr(stt), C.byref(st))
        _lib.check(s, allow=(0, 5))
        return ev, rs, it, stt, st.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            self._lib.bbl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class SolveResult:
    evals: np.ndarray
    evecs: object
    resid: np.ndarray
    stats: dict
    status: str

    @property
    def converged(self) -> bool:
        return self.status == "BBL_OK"


def solve(A: Matrix, nev: int, b: int, pivot=None, evecs: str = "device", **opts) -> SolveResult:
    """Block Lanczos for the nev lowest eigenpairs (bbl_solve).

    pivot: None (random), a CUDA tensor or a numpy array, n x b FP64.
    evecs: "device" (CUDA tensor), "host" (numpy array), "pinned" (page-locked
    CPU tensor: the copy back runs at the host link's full rate) or None."""
    torch = _torch()
    o = options(**opts)
    if "storage" not in opts:
        o.storage = FP32 if A.storage == "fp32" else FP64
    if "stream" not in opts:
        o.stream = _stream(None)
    ev = np.zeros(nev)
    rs = np.zeros(nev)
    if evecs == "device":
        X = torch.empty((A.n, nev), dtype=torch.float64, device="cuda")
    elif evecs == "host":
        X = np.zeros((A.n, nev))
    elif evecs == "pinned":
        X = torch.empty((A.n, nev), dtype=torch.float64, pin_memory=True)
    else:
        X = None
    if isinstance(pivot, np.ndarray):
        pivot = np.ascontiguousarray(pivot, dtype=np.float64)
    st = Stats()
    s = A._lib.bbl_solve(A.handle, nev, b, _ptr(pivot), C.byref(o), _ptr(ev), _ptr(X), _ptr(rs), C.byref(st))
    _lib.check(s, allow=(0, 5))
    return SolveResult(ev, X, rs, st.as_dict(), _lib.STATUS[s])

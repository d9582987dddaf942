"""ctypes declarations of the C ABI in include/bbl.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

BBL_OK = 0
STATUS = {0: "BBL_OK", 1: "BBL_ERR_INVALID_ARG", 2: "BBL_ERR_NOT_SYMMETRIC", 3: "BBL_ERR_OOM", 4: "BBL_ERR_CUDA",
          5: "BBL_ERR_NOT_CONVERGED", 6: "BBL_ERR_NUMERICAL", 7: "BBL_ERR_TIMEOUT", 8: "BBL_ERR_UNSUPPORTED"}
FP64, FP32 = 0, 1
CSR, SELL, KRON, TILED = 0, 1, 2, 3


class Options(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_vectors", C.c_int), ("criterion", C.c_int), ("rms_tol", C.c_double),
                ("seed", C.c_uint64), ("defl_tol", C.c_double), ("storage", C.c_int), ("polish", C.c_int),
                ("stage1_tol", C.c_double), ("check_every", C.c_int), ("stream", C.c_void_p),
                ("ritz_overlap", C.c_int), ("half_first_pass", C.c_int), ("restart_keep", C.c_int),
                ("max_blocks", C.c_int), ("fused_update_gram", C.c_int), ("narrow_old_updates", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("vec_equiv_iters", C.c_int), ("polish_iters", C.c_int), ("deflations", C.c_int),
                ("converged", C.c_int), ("t_spmm_ms", C.c_double), ("t_reorth_ms", C.c_double),
                ("t_cholqr_ms", C.c_double), ("t_ritz_ms", C.c_double), ("t_other_ms", C.c_double),
                ("t_total_ms", C.c_double), ("spmm_bytes", C.c_double), ("spmm_gbs", C.c_double),
                ("ns_per_op", C.c_double), ("ortho_err", C.c_double), ("spmm_bytes_total", C.c_double),
                ("reorth_bytes_total", C.c_double), ("ritz_solves", C.c_int), ("gram_calls", C.c_int),
                ("t_gram_ms", C.c_double), ("gram_bytes_total", C.c_double), ("spmm_calls", C.c_int),
                ("restarts", C.c_int), ("graph_kernels", C.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int
D = C.c_double
ST = C.c_int

# name: (restype, argtypes)
SIGNATURES = {
    "bbl_options_default": (None, [C.POINTER(Options)]),
    "bbl_last_error": (C.c_char_p, []),
    "bbl_status_string": (C.c_char_p, [ST]),
    "bbl_version": (C.c_int, []),
    "bbl_kernel_launches": (C.c_uint64, []),
    "bbl_probe_fma_rate": (ST, [I32, C.POINTER(D), P]),
    "bbl_workspace_bytes": (C.c_size_t, []),
    "bbl_workspace_release": (ST, []),
    "bbl_matrix_create": (ST, [I64, I64, P, P, P, I32, I32, I32, I32, I32, I32, P, C.POINTER(P)]),
    "bbl_matrix_create_kron": (ST, [I64, I64, I32, P, P, P, P, P, I32, I32, P, C.POINTER(P)]),
    "bbl_matrix_destroy": (None, [P]),
    "bbl_matrix_info": (ST, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(D), C.POINTER(I64), C.POINTER(I32),
                             C.POINTER(I32), C.POINTER(I64)]),
    "bbl_matrix_diagonal": (ST, [P, P, P]),
    "bbl_matrix_set_spmm_lanes": (ST, [P, I32]),
    "bbl_spmm": (ST, [P, I32, P, P, P]),
    "bbl_spmm_f64": (ST, [P, I32, P, P, P]),
    "bbl_spmm_group": (ST, [P, I32, P, P, I32, P]),
    "bbl_block_reorth": (ST, [I64, I32, I32, I32, P, P, P, I32, P]),
    "bbl_cholqr2": (ST, [I64, I32, I32, P, P, D, C.POINTER(I32), P]),
    "bbl_ritz_banded": (ST, [I32, I32, I32, P, P, P, P]),
    "bbl_ritz_vectors": (ST, [I64, I32, I32, I32, P, I32, P, P, P]),
    "bbl_pivot_random": (ST, [I64, I32, C.c_uint64, P, P]),
    "bbl_pivot_bootstrap": (ST, [P, I64, I32, D, C.c_uint64, P, P]),
    "bbl_solve": (ST, [P, I32, I32, P, C.POINTER(Options), P, P, P, C.POINTER(Stats)]),
    "bbl_block_gram": (ST, [I64, I32, I32, I32, P, P, P, P]),
    "bbl_block_gram_noalloc": (ST, [I64, I32, I32, I32, P, P, P, P]),
    "bbl_block_gram_f16": (ST, [I64, I32, P, P, P, P]),
    "bbl_block_update_gram": (ST, [I64, I32, P, P, P, P, P]),
    "bbl_block_update_f16old": (ST, [I64, I32, I32, P, P, P, P, P]),
    "bbl_pivot_rr_residual": (ST, [P, I32, P, P, P, P]),
    "bbl_pivot_overlap": (ST, [I64, I32, P, I32, P, P, P]),
    "bbl_mlp_create": (ST, [I32, I32, C.POINTER(P)]),
    "bbl_mlp_destroy": (None, [P]),
    "bbl_mlp_num_params": (C.c_int, [P]),
    "bbl_mlp_set_params": (ST, [P, P, P]),
    "bbl_mlp_get_params": (ST, [P, P, P, P]),
    "bbl_mlp_forward": (ST, [P, I32, P, P, P]),
    "bbl_mlp_loss_grad": (ST, [P, I32, P, P, C.POINTER(C.c_float), P]),
    "bbl_mlp_adam_step": (ST, [P, C.c_float, P]),
    "bbl_mlp_train": (ST, [P, I32, P, P, I32, C.c_float, P, P]),
    "bbl_pivot_learned": (ST, [P, C.c_float, I64, I32, I32, P, I32, P, P]),
    "bbl_batch_create": (ST, [I32, P, I64, P, P, P, I32, I32, I32, I32, P, C.POINTER(P)]),
    "bbl_batch_destroy": (None, [P]),
    "bbl_batch_matrix": (ST, [P, C.POINTER(P)]),
    "bbl_batch_set_schedule": (ST, [P, I32]),
    "bbl_batch_solve": (ST, [P, I32, I32, C.POINTER(Options), I32, P, P, P, P, C.POINTER(Stats)]),
}

_lib = None


def load(auto_build: bool = True):
    """Loads libbbl.so (building it first if needed).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if auto_build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libbbl.so not found at {_build.LIB}; run paper_2210_15763_gb300.build.build()")
    lib = C.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(SIGNATURES)


class BBLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, allow=(BBL_OK,)) -> int:
    if status not in allow:
        raise BBLError(status, load(False).bbl_last_error().decode(errors="replace"))
    return status

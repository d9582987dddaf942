"""Host-side checks (no GPU): the library builds, loads, and exports every
entry point include/bbl.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "bbl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:bbl_status|void|int|size_t|uint64_t|const char\*)\s+(bbl_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = header_functions()
    for f in ("bbl_matrix_create", "bbl_spmm", "bbl_pivot_bootstrap", "bbl_solve", "bbl_cholqr2",
              "bbl_block_reorth", "bbl_ritz_banded"):
        assert f in names


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2210_15763_gb300 import _lib
    from paper_2210_15763_gb300 import build as B
    B.build()
    lib = ctypes.CDLL(B.LIB)
    missing = [f for f in header_functions() if not hasattr(lib, f)]
    assert not missing, missing
    # and the binding declares each of them with the same name
    assert set(header_functions()) <= set(_lib.SIGNATURES)


def test_binding_refuses_to_run_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2210_15763_gb300 as bbl
    import synth
    with pytest.raises(RuntimeError):
        bbl.Matrix(synth.laplacian_1d(10))

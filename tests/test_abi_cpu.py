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


def _header_struct_fields(name):
    """(C type, field) pairs of `typedef struct { ... } name;` in bbl.h, in order."""
    src = open(os.path.join(ROOT, "include", "bbl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src, flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        first, *more = [d.strip() for d in decl.split(",")]  # "double a, b, c"
        ctype, _, field = first.rpartition(" ")
        ctype = ctype.replace(" *", "*")
        for f in [field] + more:
            fields.append((ctype, f.lstrip("*")))
    return fields


@pytest.mark.parametrize("cname,pyname", [("bbl_options", "Options"), ("bbl_stats", "Stats")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes mirrors of the option and statistics structs list the
    header's fields in the header's order with the same sizes, so that a
    field added on one side only cannot shift the others."""
    import ctypes as C
    from paper_2210_15763_gb300 import _lib
    size = {"double": 8, "int": 4, "unsigned long long": 8, "uint64_t": 8, "int64_t": 8, "void*": 8,
            "bbl_dtype": 4, "bbl_format": 4}
    hdr = _header_struct_fields(cname)
    py = getattr(_lib, pyname)._fields_
    assert [f for _, f in hdr] == [f for f, _ in py]
    for (ctype, field), (_, pytype) in zip(hdr, py):
        assert ctype in size, (field, ctype)
        assert size[ctype] == C.sizeof(pytype), (field, ctype, pytype)

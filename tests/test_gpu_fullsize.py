"""Full-size parity: the n = 2,000,000 synthetic Kronecker workloads (about
300 and 200 nonzeros per row) against the FP64 oracle's eigenvalues stored
by tests/golden/make_reference_evals.py (plain FP64 block Lanczos, b = 8,
splitmix64 random pivot, seed 20221028, residual 1e-8 * ||H||_inf).

FP64 solve: same pivot, the eight eigenvalues to relative 1e-10, the same
block count (+-1).  Mixed precision (FP32 stage + polish): relative 1e-10.
FP32 stage alone (no polish, stage tolerance 2e-6): relative error <= 1e-6
for every eigenvalue (the mixed-precision bar), reported per eigenvalue.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import rng as OR
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}_fp64_oracle_evals.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle eigenvalues for {name}")
    with open(path) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def kron_n2e6():
    return synth.kron_matrix("kron_n2e6")


def test_fullsize_fp64_solve_matches_oracle(kron_n2e6):
    torch, bbl = need_gpu()
    ref = _golden("kron_n2e6")
    A = kron_n2e6
    assert A.n == ref["n"] and A.nnz == ref["nnz"]
    M = bbl.Matrix(A, storage="fp64")
    piv = OR.normal_block(ref["pivot_seed"], A.n, ref["b"])
    r = bbl.solve(M, ref["nev"], ref["b"], pivot=piv, tol=ref["tol"], check_every=1, max_vectors=2000, evecs=None)
    M.close()
    assert r.converged
    np.testing.assert_allclose(r.evals, ref["evals"], rtol=1e-10)
    assert abs(r.stats["iters"] - ref["blocks"]) <= 1
    assert np.all(r.resid <= ref["tol"] * ref["norm_inf"] * 1.01)


def test_fullsize_mixed_precision_matches_oracle(kron_n2e6):
    torch, bbl = need_gpu()
    ref = _golden("kron_n2e6")
    A = kron_n2e6
    M = bbl.Matrix(A, storage="fp32", fmt="csr")
    piv = OR.normal_block(ref["pivot_seed"], A.n, ref["b"])
    r = bbl.solve(M, ref["nev"], ref["b"], pivot=piv, tol=ref["tol"], max_vectors=2000, evecs=None)
    assert r.converged
    np.testing.assert_allclose(r.evals, ref["evals"], rtol=1e-10)
    assert np.all(r.resid <= ref["tol"] * ref["norm_inf"] * 1.01)
    # the FP32 stage on its own (no polish): every eigenvalue within 1e-6
    r1 = bbl.solve(M, ref["nev"], ref["b"], pivot=piv, tol=2e-6, polish=0, max_vectors=2000, evecs=None)
    M.close()
    rel = np.abs(r1.evals - np.array(ref["evals"])) / np.abs(ref["evals"])
    print("FP32-stage relative eigenvalue errors vs the FP64 oracle:", " ".join(f"{x:.2e}" for x in rel))
    assert rel.max() <= 1e-6, rel


@pytest.mark.parametrize("fmt,sigma", [("sell", 1024), ("csr", 0), ("tiled", 1000)])
def test_fullsize_headline_step_matches_oracle(kron_n2e6, fmt, sigma):
    """The benchmark's timed step exactly: the bootstrapped pivot (20,000
    lowest-diagonal rows, truncated-space sub-solve to 1e-4 in FP32 storage),
    the FP32 stage to 3e-7 with the FP16 first-pass Gram, the float-float
    polish and the FP64 residuals, on the FP32-stored matrix in each format
    the SpMM autotuner may pick (SELL-C-sigma with sigma = 1024, CSR, or
    the tiled format with tiles of 1000).
    The eight eigenvalues agree with the FP64 oracle's to relative 1e-10."""
    import bench
    torch, bbl = need_gpu()
    ref = _golden("kron_n2e6")
    A = kron_n2e6
    M = bbl.Matrix(A, storage="fp32", fmt=fmt, sell_sigma=sigma)
    P = bench.headline_pivot(bbl, M)
    r = bench.headline_solve(bbl, M, P, evecs=None)
    M.close()
    assert r.converged
    rel = np.abs(r.evals - np.array(ref["evals"])) / np.abs(ref["evals"])
    print(f"headline step ({fmt}) relative eigenvalue errors vs the FP64 oracle:", " ".join(f"{x:.2e}" for x in rel))
    assert rel.max() <= 1e-10, rel
    assert bench.oracle_eval_error(r.evals) == pytest.approx(rel.max())
    assert np.all(r.resid <= ref["tol"] * ref["norm_inf"] * 1.01)


def test_fullsize_c3_family_mixed_precision_error_table():
    """The ~200 nonzeros-per-row family (K = 12, c = 3.9) at n = 2e6: the
    FP32 stage's per-eigenvalue error against the FP64 oracle (<= 1e-6) and
    the polished result (1e-10)."""
    torch, bbl = need_gpu()
    ref = _golden("kron_n2e6_c3")
    A = synth.kron_matrix("kron_n2e6_c3")
    assert A.n == ref["n"] and A.nnz == ref["nnz"]
    M = bbl.Matrix(A, storage="fp32", fmt="sell", sell_sigma=256)
    piv = OR.normal_block(ref["pivot_seed"], A.n, ref["b"])
    r1 = bbl.solve(M, ref["nev"], ref["b"], pivot=piv, tol=2e-6, polish=0, max_vectors=2000, evecs=None)
    rel = np.abs(r1.evals - np.array(ref["evals"])) / np.abs(ref["evals"])
    print("FP32-stage relative eigenvalue errors vs the FP64 oracle:", " ".join(f"{x:.2e}" for x in rel))
    assert rel.max() <= 1e-6, rel
    r = bbl.solve(M, ref["nev"], ref["b"], pivot=piv, tol=ref["tol"], max_vectors=2000, evecs=None)
    M.close()
    assert r.converged
    np.testing.assert_allclose(r.evals, ref["evals"], rtol=1e-10)

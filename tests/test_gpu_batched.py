"""Batched form: many uneven problems in one graph launch, against dense
eigensolves and against the single-problem solver."""
import numpy as np
import pytest

import synth
from oracle import rng as OR
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _family(count=7, seed=3):
    mats = []
    rng = np.random.default_rng(seed)
    for s in range(count):
        nP = int(rng.integers(24, 48))
        nN = int(rng.integers(20, 36))
        f = synth.kron_factors(nP, nN, K=4, c=3.0, seed=100 + s)
        mats.append(synth.assemble(f))
    return mats


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_batched_solve_matches_dense_eigensolves(storage):
    torch, bbl = need_gpu()
    mats = _family()
    B = bbl.Batch(mats, storage=storage)
    tol = 1e-10 if storage == "fp64" else 1e-6
    ev, rs, it, st, stats = B.solve(4, 4, use_graph=True, tol=tol, max_vectors=400, seed=11)
    assert np.all(st == 0), st
    for s, A in enumerate(mats):
        want = np.linalg.eigvalsh(A.to_dense())[:4]
        rel = 1e-10 if storage == "fp64" else 1e-5
        np.testing.assert_allclose(ev[s], want, rtol=rel, atol=rel * np.abs(want).max())
    nrm = np.array([np.abs(A.to_dense()).sum(axis=1).max() for A in mats])
    assert np.all(rs.max(axis=1) <= (1e-8 if storage == "fp64" else 1e-4) * nrm)


@pytest.mark.parametrize("storage,b", [("fp64", 2), ("fp64", 8), ("fp32", 8), ("fp32", 16)])
def test_batched_block_sizes_match_dense_eigensolves(storage, b):
    """Other block sizes: b = 8 and 16 take the row-contiguous segmented Gram
    (tile-sized chunks), b = 2 the column-group one.  The FP64 oracle needs
    up to 47 blocks of 8 on these matrices at 1e-10, so the basis may hold
    640 vectors (capped per problem by the smallest one's size)."""
    torch, bbl = need_gpu()
    mats = _family(count=5, seed=17)
    B = bbl.Batch(mats, storage=storage)
    tol = 1e-10 if storage == "fp64" else 2e-6
    ev, rs, it, st, stats = B.solve(4, b, tol=tol, max_vectors=640, seed=5)
    assert np.all(st == 0), st
    rel = 1e-10 if storage == "fp64" else 1e-5
    for s, A in enumerate(mats):
        want = np.linalg.eigvalsh(A.to_dense())[:4]
        np.testing.assert_allclose(ev[s], want, rtol=rel, atol=rel * np.abs(want).max())


def test_batched_graph_and_host_loop_agree():
    torch, bbl = need_gpu()
    mats = _family(count=5, seed=8)
    B = bbl.Batch(mats, storage="fp64")
    e1, r1, i1, s1, _ = B.solve(4, 4, use_graph=True, tol=1e-9, max_vectors=120, seed=2)
    e2, r2, i2, s2, _ = B.solve(4, 4, use_graph=False, tol=1e-9, max_vectors=120, seed=2)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(e1, e2)


def test_batched_adaptive_tests_stop_at_or_just_after_every_block_tests():
    """Per-problem adaptive test schedule against a test after every block:
    a problem can only stop at a tested block, so it stops at or after the
    first block that passes, within the 8-block step bound; the eigenvalues
    agree to the tolerance either way."""
    torch, bbl = need_gpu()
    mats = _family(count=6, seed=12)
    B = bbl.Batch(mats, storage="fp64")
    # the FP64 oracle needs 44-64 blocks of 4 on these matrices at 1e-9
    e1, r1, i1, s1, _ = B.solve(4, 4, tol=1e-9, max_vectors=400, seed=4, check_every=1)
    e0, r0, i0, s0, _ = B.solve(4, 4, tol=1e-9, max_vectors=400, seed=4, check_every=0)
    assert np.all(s1 == 0) and np.all(s0 == 0), (s1, s0)
    assert np.all(i0 >= i1) and np.all(i0 <= i1 + 8), (i0, i1)
    nrm = np.array([np.abs(A.to_dense()).sum(axis=1).max() for A in mats])
    np.testing.assert_allclose(e0, e1, rtol=0, atol=1e-8 * nrm.max())
    assert np.all(r0.max(axis=1) <= 1e-7 * nrm)


def test_batched_segment_equals_single_solve_with_the_same_pivot():
    torch, bbl = need_gpu()
    mats = _family(count=4, seed=5)
    B = bbl.Batch(mats, storage="fp64")
    ev, rs, it, st, _ = B.solve(4, 4, tol=1e-9, max_vectors=120, seed=21)
    # the batched pivot is the splitmix64 normal block over the stacked rows
    P = OR.normal_block(21, B.n, 4)
    for s in (0, 2):
        o0, o1 = B.offsets[s], B.offsets[s + 1]
        r = bbl.solve(bbl.Matrix(mats[s]), 4, 4, pivot=P[o0:o1].copy(), tol=1e-9, max_vectors=120)
        np.testing.assert_allclose(ev[s], r.evals, rtol=1e-10)
        assert abs(int(it[s]) - r.stats["iters"]) <= 1


def test_batched_fp32_polish_reaches_the_fp64_tolerance():
    """FP32 blocks alone stop at their floor, far above 1e-10; with the
    polish (default) the problems that miss the tolerance go on from their
    FP32 Ritz vectors with FP64 blocks, and every problem then matches the
    dense eigenvalues to 1e-10 with true FP64 residuals <= tol * ||H_s||."""
    torch, bbl = need_gpu()
    mats = _family(count=6, seed=9)
    B = bbl.Batch(mats, storage="fp32")
    tol = 1e-10
    e0, r0, i0, s0, _ = B.solve(4, 4, tol=tol, max_vectors=400, seed=3, polish=0)
    assert np.any(s0 != 0)
    ev, rs, it, st, stats = B.solve(4, 4, tol=tol, max_vectors=400, seed=3)
    assert np.all(st == 0), st
    assert stats["polish_iters"] >= 1
    nrm = np.array([np.abs(A.to_dense()).sum(axis=1).max() for A in mats])
    for s, A in enumerate(mats):
        want = np.linalg.eigvalsh(A.to_dense())[:4]
        np.testing.assert_allclose(ev[s], want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
        assert np.all(rs[s] <= tol * nrm[s] * (1 + 1e-6))
    assert np.all(it >= i0)


def test_batched_rejects_coupled_segments():
    torch, bbl = need_gpu()
    a = synth.random_sparse_symmetric(40, 4, seed=1)
    b = synth.random_sparse_symmetric(30, 4, seed=2)
    offsets, rp, col, val = bbl.stack_block_diagonal([a, b])
    col = col.copy()
    col[0] = 60  # row 0 (segment 0) references a column of segment 1
    from paper_2210_15763_gb300 import _lib
    import ctypes as C
    lib = _lib.load()
    h = C.c_void_p()
    st = lib.bbl_batch_create(2, offsets.ctypes.data_as(C.c_void_p), int(rp[-1]), rp.ctypes.data_as(C.c_void_p),
                              col.ctypes.data_as(C.c_void_p), val.ctypes.data_as(C.c_void_p), 0, 0, 0, 0, None,
                              C.byref(h))
    assert _lib.STATUS[st] == "BBL_ERR_INVALID_ARG"


def test_autotuner_picks_a_valid_schedule_and_caches_it(tmp_path, monkeypatch):
    torch, bbl = need_gpu()
    from paper_2210_15763_gb300 import autotune
    monkeypatch.setenv("BBL_AUTOTUNE_CACHE", str(tmp_path / "t.json"))
    A = synth.kron_matrix("kron_n2e4", scale=0.5)
    best = autotune.tune(A, 4, storage="fp32", reps=2)
    assert best["fmt"] in ("csr", "sell") and not best["cached"]
    assert best["ms"] == min(t["ms"] for t in best["timings"])
    again = autotune.tune(A, 4, storage="fp32", reps=2)
    assert again["cached"] and again["fmt"] == best["fmt"]

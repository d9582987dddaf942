"""Plants plausible mistakes in the oracle (on the CPU) and checks that the
pins notice: a transposed off-diagonal block of T, the garbled Eq. 7 taken
literally, a wrong sign in the Gram-Schmidt subtraction, and a dropped
reorthogonalisation."""
import numpy as np

import synth
from oracle import lanczos as L
from oracle import rng as R


def _dense_pin_error():
    """Relative eigenvalue error of block Lanczos (b = 3) against a dense solve."""
    A = synth.random_sparse_symmetric(90, 6, seed=4)
    want = np.linalg.eigvalsh(A.to_dense())[:5]
    r = L.block_lanczos(A, 5, 3, R.normal_block(3, A.n, 3), tol=1e-11, max_vectors=90)
    return np.max(np.abs(r.evals - want) / np.abs(want))


def _orthonormality_error():
    H = synth.kron_matrix("kron_n2e4", scale=0.15)
    r = L.block_lanczos(H, 4, 3, R.normal_block(6, H.n, 3), tol=1e-9, keep_basis=True)
    return np.max(np.abs(r.V.T @ r.V - np.eye(r.V.shape[1])))


def _fails(fn, bound):
    """True when the pin no longer holds: an error above `bound`, NaN, or an exception."""
    try:
        with np.errstate(all="ignore"):
            err = fn()
    except (FloatingPointError, np.linalg.LinAlgError, ValueError):
        return True
    return not (err <= bound)


def test_unmodified_oracle_passes_both_pins():
    assert _dense_pin_error() < 1e-10
    assert _orthonormality_error() < 1e-12


def test_transposed_offdiagonal_block_is_caught(monkeypatch):
    orig = L.block_tridiagonal
    monkeypatch.setattr(L, "block_tridiagonal", lambda A, B: orig(A, [x.T for x in B]))
    assert _fails(_dense_pin_error, 1e-10)


def test_eq7_taken_literally_is_caught():
    # The loop of block_lanczos written out with A_n = W^T W (Eq. 7 as printed)
    # instead of V_n^T W: the Ritz values no longer match the dense solve.
    A = synth.random_sparse_symmetric(90, 6, seed=4)
    want = np.linalg.eigvalsh(A.to_dense())[:5]
    H = A.to_scipy()
    V = [np.linalg.qr(R.normal_block(3, A.n, 3))[0]]
    As, Bs = [], []
    for j in range(20):
        W = H @ V[j]
        Aj = W.T @ W
        W = W - V[j] @ Aj
        if j:
            W = W - V[j - 1] @ Bs[j - 1].T
        Q = np.hstack(V)
        W = L.cgs_pass(L.cgs_pass(W, Q), Q)
        Vn, Bj, _ = L.cholqr2(W, 0.0)
        As.append(Aj)
        V.append(Vn)
        Bs.append(Bj)
    theta = np.linalg.eigvalsh(L.block_tridiagonal(As, Bs[:-1]))[:5]
    assert np.max(np.abs(theta - want) / np.abs(want)) > 1e-3


def test_wrong_sign_in_gram_schmidt_is_caught(monkeypatch):
    monkeypatch.setattr(L, "cgs_pass", lambda W, Q: W if Q is None or Q.shape[1] == 0 else W + Q @ (Q.T @ W))
    assert _fails(_orthonormality_error, 1e-12)


def test_dropped_reorthogonalisation_is_caught(monkeypatch):
    monkeypatch.setattr(L, "cgs_pass", lambda W, Q: W)
    assert _fails(_orthonormality_error, 1e-12)


def test_thick_restart_without_the_coupling_is_caught(monkeypatch):
    # the restart's coupling C between the kept Ritz vectors and the newest
    # block dropped from the projected matrix: the restarted runs no longer
    # reach the dense spectrum
    A = synth.random_sparse_symmetric(300, 6, seed=34)
    want = np.linalg.eigvalsh(A.to_dense())[:4]
    orig = L.restarted_projection
    monkeypatch.setattr(L, "restarted_projection", lambda th, C, As, Bs: orig(th, 0.0 * C, As, Bs))

    def err():
        r = L.block_lanczos_thick(A, 4, 4, R.normal_block(2, A.n, 4), tol=1e-10, max_vectors=24, keep=8,
                                  max_blocks=400)
        return np.max(np.abs(r.evals - want) / np.abs(want)) if r.converged else np.inf

    assert _fails(err, 1e-10)

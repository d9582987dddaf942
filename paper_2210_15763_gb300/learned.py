"""Learned pivot for a family H(g): driver over the library's entry points.

Training data are the method's own solves: for each training parameter g,
the bootstrapped pivot (Sec. II.B) and a block Lanczos solve give the lowest
eigenvectors X(g).  The eigenvectors at `n_basis_g` evenly spaced training
values are orthonormalised block by block (CGS2 + CholQR2 on the GPU) into
the stored basis U (FP32, nbasis = n_basis_g * nev columns).  The network
is trained to map g to the coefficients C(g) = U^T X(g) (FP64 Gram on the
GPU).  At inference P = U f(g); Lanczos still decides: the learned pivot
is used only if the Rayleigh-Ritz residual of its span is below that of
every bootstrapped pivot seen in training (else the bootstrapped pivot is
built and the better of the two taken), and a solve that does not converge
is restarted from the bootstrapped pivot.

Every numerical step runs in libbbl.so; this module sequences the calls.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import Matrix, MLP, block_gram, block_reorth, cholqr2, pivot_bootstrap, pivot_rr_residual, solve


def init_params(hidden: int, out_dim: int, seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (packed FP32)."""
    r = np.random.default_rng(seed)
    parts = []
    for o, i in ((hidden, 1), (hidden, hidden), (out_dim, hidden)):
        lim = 1.0 / math.sqrt(i)
        parts.append(r.uniform(-lim, lim, size=o * i).astype(np.float32))
        parts.append(np.zeros(o, dtype=np.float32))
    return np.concatenate(parts)


@dataclasses.dataclass
class LearnedPivot:
    mlp: MLP
    U: object          # (nblocks, n, nev) FP32 CUDA tensor
    nev: int
    g_train: np.ndarray
    loss: np.ndarray
    train_iters: list
    rr_boot_train: float = float("inf")  # smallest Rayleigh-Ritz residual of a training bootstrap pivot

    def pivot(self, g: float):
        return self.mlp.pivot(g, self.U, self.nev)


def fit(make_matrix, g_train, nev: int, b: int, trunc_dim: int, n_basis_g: int = 8, hidden: int = 128,
        epochs: int = 3000, lr: float = 1e-3, seed: int = 0, tol: float = 1e-8, storage: str = "fp32",
        fmt: str = "sell", sub_tol: float = 1e-4) -> LearnedPivot:
    """make_matrix(g) -> host CSR; solves H(g) for every training g from the
    bootstrapped pivot (truncated-space sub-solve to sub_tol)."""
    import torch
    g_train = np.asarray(g_train, dtype=np.float64)
    X, iters, rr_boot = [], [], []
    for g in g_train:
        M = Matrix(make_matrix(g), storage=storage, fmt=fmt, sell_sigma=256 if fmt == "sell" else 0)
        P = pivot_bootstrap(M, trunc_dim, b, sub_tol=sub_tol, seed=seed)
        _, rb = pivot_rr_residual(M, P)
        rr_boot.append(float(np.max(rb[:min(nev, rb.size)])))
        r = solve(M, nev, b, pivot=P, tol=tol)
        X.append(r.evecs)
        iters.append(r.stats["iters"] + r.stats["polish_iters"])
        M.close()
    n = X[0].shape[0]
    # stored basis: eigenvectors at n_basis_g evenly spaced training values, orthonormalised
    order = np.argsort(g_train)
    pick = order[np.round(np.linspace(0, len(order) - 1, n_basis_g)).astype(int)]
    blocks = []
    for k in pick:
        Z = X[k].clone()
        if blocks:
            block_reorth(torch.stack(blocks), Z, passes=2)
        cholqr2(Z)
        blocks.append(Z)
    U64 = torch.stack(blocks)                       # (n_basis_g, n, nev) FP64
    U = U64.to(torch.float32).contiguous()
    # targets C(g) = U^T X(g), flattened row-major (nbasis x nev)
    T = torch.stack([block_gram(U64, Xg).reshape(-1) for Xg in X]).to(torch.float32).contiguous()
    out_dim = T.shape[1]
    net = MLP(hidden, out_dim)
    net.set_params(init_params(hidden, out_dim, seed))
    gd = torch.tensor(g_train, dtype=torch.float32, device="cuda")
    loss = net.train(gd, T, epochs, lr)
    return LearnedPivot(net, U, nev, g_train, loss, iters, float(np.min(rr_boot)))


def rr_max(A: Matrix, P, nev: int) -> float:
    """Largest Rayleigh-Ritz residual of the nev lowest pairs of span(P) (one SpMM)."""
    _, r = pivot_rr_residual(A, P)
    return float(np.max(r[:min(nev, r.size)]))


def solve_with_learned_pivot(A: Matrix, lp: LearnedPivot, g: float, b: int, trunc_dim: int, tol: float = 1e-8,
                             seed: int = 0, sub_tol: float = 1e-4):
    """Lanczos decides on the learned pivot (one Rayleigh-Ritz SpMM).  When
    its residual is below every bootstrapped pivot's seen in training, it is
    used at once; otherwise the bootstrapped pivot is built (sub-solve to
    sub_tol) and the one with the smaller residual taken (one more SpMM).  A
    solve from the learned pivot that does not converge is redone from the
    bootstrapped pivot."""
    P_l = lp.pivot(g)
    rl = rr_max(A, P_l, lp.nev)
    P_b, rb = None, None
    if rl < lp.rr_boot_train:
        P, used = P_l, True
    else:
        P_b = pivot_bootstrap(A, trunc_dim, b, sub_tol=sub_tol, seed=seed)
        rb = rr_max(A, P_b, lp.nev)
        used = rl <= rb
        P = P_l if used else P_b
    r = solve(A, lp.nev, b, pivot=P, tol=tol)
    fallback = False
    if not r.converged and used:
        if P_b is None:
            P_b = pivot_bootstrap(A, trunc_dim, b, sub_tol=sub_tol, seed=seed)
        r = solve(A, lp.nev, b, pivot=P_b, tol=tol)
        fallback = True
    return r, {"learned_used": used, "rr_learned": rl, "rr_boot": rb, "fallback": fallback,
               "bootstrap_built": P_b is not None}

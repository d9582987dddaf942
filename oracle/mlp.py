"""Learned-pivot MLP in FP64 (oracle; test infrastructure only).

The paper has no learned component; this is the reference for the GPU
training and inference kernels of the learned-pivot form.  Network:

    h1 = gelu(W1 g + b1)         1 -> H1
    h2 = gelu(W2 h1 + b2)        H1 -> H2
    y  = W3 h2 + b3              H2 -> 64 * b  (coefficients on the basis U)

gelu(x) = x/2 (1 + erf(x / sqrt 2)) (exact form).  Weight matrices are
stored out x in (row-major).  `bf16_round` rounds weights to bfloat16
(round to nearest even) so that the oracle sees the same weights the GPU
forward pass uses; arithmetic here is FP64.

Loss: mean over the batch and outputs of (y - target)^2.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
import math

import numpy as np

PARAMS = ("W1", "b1", "W2", "b2", "W3", "b3")


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Rounds FP32 values to bfloat16 (nearest, ties to even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _erf(x):
    return np.vectorize(math.erf)(x)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def init_params(out_dim: int, hidden: int = 128, seed: int = 0) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, FP32-rounded."""
    r = np.random.default_rng(seed)
    dims = [(hidden, 1), (hidden, hidden), (out_dim, hidden)]
    p = {}
    for k, (o, i) in enumerate(dims, start=1):
        lim = 1.0 / math.sqrt(i)
        p[f"W{k}"] = r.uniform(-lim, lim, size=(o, i)).astype(np.float32).astype(np.float64)
        p[f"b{k}"] = np.zeros(o)
    return p


def forward(p: dict, g: np.ndarray, bf16_weights: bool = True):
    """Returns (y, cache); g has shape (batch,)."""
    W = {k: (bf16_round(p[k]) if bf16_weights else p[k]) for k in ("W1", "W2", "W3")}
    x0 = np.asarray(g, dtype=np.float64).reshape(-1, 1)
    z1 = x0 @ W["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ W["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ W["W3"].T + p["b3"]
    return y, dict(x0=x0, z1=z1, h1=h1, z2=z2, h2=h2, W=W)


def loss_and_grads(p: dict, g: np.ndarray, target: np.ndarray, bf16_weights: bool = True):
    """MSE loss and its gradients by hand-written back-propagation."""
    y, c = forward(p, g, bf16_weights)
    N = y.size
    diff = y - target
    loss = float(np.sum(diff * diff) / N)
    dy = 2.0 * diff / N
    W = c["W"]
    gr = {}
    gr["W3"] = dy.T @ c["h2"]
    gr["b3"] = dy.sum(axis=0)
    dh2 = dy @ W["W3"]
    dz2 = dh2 * gelu_grad(c["z2"])
    gr["W2"] = dz2.T @ c["h1"]
    gr["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ W["W2"]
    dz1 = dh1 * gelu_grad(c["z1"])
    gr["W1"] = dz1.T @ c["x0"]
    gr["b1"] = dz1.sum(axis=0)
    return loss, gr


def adam_step(p: dict, gr: dict, state: dict, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in PARAMS:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1.0 - beta1) * gr[k]
        v[...] = beta2 * v + (1.0 - beta2) * gr[k] * gr[k]
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)

"""Learned-pivot form: the MLP kernels against the FP64 oracle, and the gain
of the trained network over the method without it on a small H(g) family.

Gradient tolerance: both sides use the same BF16-rounded weights; the GPU
accumulates in FP32 over at most 512 terms per sum, so agreement to relative
1e-3 of the largest gradient entry is required (FP32 round-off ~1e-6 per
operation, amplified by cancellation)."""
import numpy as np
import pytest

import synth
from oracle import mlp as OM
from tests.gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu
PN = ("W1", "b1", "W2", "b2", "W3", "b3")


def pack(p):
    return np.concatenate([p[k].reshape(-1) for k in PN]).astype(np.float32)


def unpack(v, H, O):
    shapes = [(H, 1), (H,), (H, H), (H,), (O, H), (O,)]
    out, o = {}, 0
    for k, s in zip(PN, shapes):
        sz = int(np.prod(s))
        out[k] = v[o:o + sz].reshape(s).astype(np.float64)
        o += sz
    return out


def _setup(H=32, O=40, batch=12, seed=0):
    p = OM.init_params(O, hidden=H, seed=seed)
    r = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        p[k] = (r.standard_normal(p[k].shape) * 0.1).astype(np.float32).astype(np.float64)
    g = r.uniform(0, 1, size=batch).astype(np.float32).astype(np.float64)
    tgt = r.standard_normal((batch, O)).astype(np.float32).astype(np.float64)
    return p, g, tgt


@pytest.mark.parametrize("H,O,batch", [(32, 40, 12), (128, 512, 48)])
def test_mlp_forward_and_gradients_match_oracle(H, O, batch):
    torch, bbl = need_gpu()
    p, g, tgt = _setup(H, O, batch)
    net = bbl.MLP(H, O)
    net.set_params(pack(p))
    gd = to_dev(torch, g, torch.float32)
    td = to_dev(torch, tgt, torch.float32)
    y = net.forward(gd).cpu().numpy()
    y_ref, _ = OM.forward(p, g, bf16_weights=True)
    np.testing.assert_allclose(y, y_ref, rtol=1e-4, atol=1e-5 * np.abs(y_ref).max())
    loss = net.loss_grad(gd, td)
    loss_ref, gr_ref = OM.loss_and_grads(p, g, tgt, bf16_weights=True)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    _, grads = net.get_params()
    gr = unpack(grads, H, O)
    for k in PN:
        scale = np.abs(gr_ref[k]).max() + 1e-30
        np.testing.assert_allclose(gr[k], gr_ref[k], rtol=0, atol=1e-3 * scale, err_msg=k)


def test_mlp_adam_step_matches_oracle():
    torch, bbl = need_gpu()
    H, O, batch = 32, 40, 12
    p, g, tgt = _setup(H, O, batch, seed=3)
    net = bbl.MLP(H, O)
    net.set_params(pack(p))
    gd = to_dev(torch, g, torch.float32)
    td = to_dev(torch, tgt, torch.float32)
    st = {}
    for _ in range(3):
        net.loss_grad(gd, td)
        net.adam_step(1e-2)
        _, gr = OM.loss_and_grads(p, g, tgt, bf16_weights=True)
        OM.adam_step(p, gr, st, lr=1e-2)
    got, _ = net.get_params()
    want = pack(p)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-4)


def test_mlp_graph_training_reduces_the_loss():
    torch, bbl = need_gpu()
    H, O, batch = 64, 64, 48
    p, _, _ = _setup(H, O, batch, seed=5)
    g = np.linspace(0, 1, batch)
    tgt = np.stack([np.sin(3 * g + k) for k in range(O)], axis=1)
    net = bbl.MLP(H, O)
    net.set_params(pack(p))
    hist = net.train(to_dev(torch, g, torch.float32), to_dev(torch, tgt, torch.float32), 800, 3e-3)
    assert hist[-1] < 0.05 * hist[0]


def test_learned_pivot_beats_random_and_bootstrap_on_held_out_parameters():
    """Train on 24 solves of H(g) = H0 + g V (n = 40 x 40), evaluate 6 held-out
    g: fewer blocks than from a random pivot and than from the bootstrapped
    pivot the method would use without the network."""
    torch, bbl = need_gpu()
    from paper_2210_15763_gb300 import learned
    h0, v = synth.learned_family(scale=0.04)        # nP = nN = 40 -> n = 1600
    make = lambda g: synth.family_matrix(h0, v, g)
    gs = synth.family_g(count=30)
    lp = learned.fit(make, gs[:24], nev=4, b=4, trunc_dim=200, n_basis_g=4, hidden=64, epochs=1500, lr=2e-3,
                     storage="fp64", fmt="csr")
    assert lp.loss[-1] < 0.2 * lp.loss[0]
    it_l, it_r, it_b = [], [], []
    for g in gs[24:]:
        A = bbl.Matrix(make(g))
        r_l, info = learned.solve_with_learned_pivot(A, lp, g, 4, 200)
        r_r = bbl.solve(A, 4, 4, pivot=None, seed=1, tol=1e-8)
        r_b = bbl.solve(A, 4, 4, pivot=bbl.pivot_bootstrap(A, 200, 4, sub_tol=1e-4), tol=1e-8)
        ref = np.linalg.eigvalsh(make(g).to_dense())[:4]
        np.testing.assert_allclose(r_l.evals, ref, rtol=1e-10)
        it_l.append(r_l.stats["iters"])
        it_r.append(r_r.stats["iters"])
        it_b.append(r_b.stats["iters"])
    assert np.mean(it_l) < np.mean(it_r), (it_l, it_r)
    assert np.mean(it_l) < np.mean(it_b), (it_l, it_b)

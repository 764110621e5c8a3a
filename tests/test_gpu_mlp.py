"""Warm-start network kernels (forward, backward, Adam) on the GPU against the
CPU oracle of the same network (BF16-rounded weights, FP64 arithmetic)."""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as mo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    return mgw.Handle(0)


@pytest.mark.parametrize("dims,batch", [((16, 256, 1), 300), ((5, 37, 3), 33)])
def test_forward_and_gradients_match_oracle(h, dims, batch):
    d_in, width, d_out = dims
    n = h.mgw_mlp_nparams(*dims)
    assert n == mo.nparams(*dims)
    g = np.random.default_rng(7)
    p = mo.init_params(*dims, seed=3)
    p[:] += 0.01 * g.standard_normal(n).astype(np.float32)  # nonzero biases too
    x = g.standard_normal((batch, d_in)).astype(np.float32)
    t = g.standard_normal((batch, d_out)).astype(np.float32)
    P = torch.from_numpy(p).cuda()
    Wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    h.mgw_mlp_round(P, Wb)
    X = torch.from_numpy(x).cuda()
    acts = torch.empty((4, batch, width), dtype=torch.float32, device="cuda")
    Y = h.mgw_mlp_forward(dims, P, Wb, X, acts=acts)
    y_ref, _ = mo.forward(p.astype(np.float64), x.astype(np.float64), *dims)
    assert np.abs(Y.cpu().numpy() - y_ref).max() <= 1e-4 * max(1.0, np.abs(y_ref).max())
    dY = torch.empty_like(Y)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    h.mgw_mlp_mse(Y, torch.from_numpy(t).cuda(), dY, loss)
    grad = torch.empty(n, dtype=torch.float32, device="cuda")
    h.mgw_mlp_backward(dims, Wb, X, acts, dY, grad)
    l_ref, g_ref = mo.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), *dims)
    assert abs(loss.item() - l_ref) <= 1e-4 * l_ref
    gr = grad.cpu().numpy()
    assert np.linalg.norm(gr - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_adam_training_on_gpu_matches_oracle_steps(h):
    dims = (3, 32, 1)
    g = np.random.default_rng(2)
    x = g.uniform(-1, 1, (128, 3)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2])[:, None].astype(np.float32)
    p = mo.init_params(*dims, seed=5)
    n = p.size
    P = torch.from_numpy(p.copy()).cuda()
    Wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    h.mgw_mlp_round(P, Wb)
    M = torch.zeros(n, dtype=torch.float32, device="cuda")
    V = torch.zeros_like(M)
    X, T = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    acts = torch.empty((4, 128, 32), dtype=torch.float32, device="cuda")
    dY = torch.empty((128, 1), dtype=torch.float32, device="cuda")
    grad = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    pr, m, v = p.copy(), np.zeros(n), np.zeros(n)
    losses = []
    for step in range(1, 201):
        Y = h.mgw_mlp_forward(dims, P, Wb, X, acts=acts)
        h.mgw_mlp_mse(Y, T, dY, loss)
        h.mgw_mlp_backward(dims, Wb, X, acts, dY, grad)
        h.mgw_mlp_adam(P, Wb, grad, M, V, step, 1e-2)
        losses.append(loss.item())
        if step <= 3:  # the first steps follow the oracle's trajectory closely
            _, gr = mo.loss_and_grad(pr.astype(np.float64), x.astype(np.float64), t.astype(np.float64), *dims)
            pr, m, v = mo.adam_step(pr, gr, m, v, step, 1e-2)
            assert np.abs(P.cpu().numpy() - pr).max() < 1e-4
    assert losses[-1] < 0.05 * losses[0]

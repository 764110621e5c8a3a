"""Pins of the warm-start network oracle: the analytic gradient against
central finite differences of the loss (with the BF16 rounding of the weights
frozen at the evaluation point), BF16 rounding against known values, and
Adam reducing the loss on a fixed regression problem."""
import numpy as np

from oracle import mlp_oracle as mo


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.0, 65504.0, 1e-3], dtype=np.float32)
    r = mo.bf16_round(x)
    # 1 + 2^-8 is a tie -> even (1.0); 1 + 1.5 * 2^-8 rounds up to 1 + 2^-7
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125 and r[3] == -3.0
    assert abs(r[4] - 65536.0) < 1e-9
    assert abs(r[5] - 1e-3) / 1e-3 < 2.0**-8


def test_gradient_against_finite_differences():
    d_in, width, d_out = 5, 16, 2
    g = np.random.default_rng(0)
    p = mo.init_params(d_in, width, d_out, 1).astype(np.float64)
    # put the weights on the BF16 grid so the rounding is locally constant
    n = mo.nparams(d_in, width, d_out)
    p = mo.bf16_round(p.astype(np.float32))
    x = g.standard_normal((7, d_in))
    t = g.standard_normal((7, d_out))
    loss, grad = mo.loss_and_grad(p, x, t, d_in, width, d_out)

    def loss_at(q):
        # rounding frozen: evaluate with unrounded weights equal to q
        W1, b1, W2, b2, W3, b3 = mo.unpack(q, d_in, width, d_out)
        a1 = mo.silu(x @ W1.T + b1)
        a2 = mo.silu(a1 @ W2.T + b2)
        y = a2 @ W3.T + b3
        return 0.5 * np.sum((y - t) ** 2) / x.shape[0]
    assert abs(loss_at(p) - loss) < 1e-12
    idx = g.choice(n, 40, replace=False)
    for i in idx:
        e = np.zeros(n)
        e[i] = 1e-6
        fd = (loss_at(p + e) - loss_at(p - e)) / 2e-6
        assert abs(fd - grad[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_adam_fits_a_smooth_target():
    d_in, width, d_out = 3, 32, 1
    g = np.random.default_rng(2)
    x = g.uniform(-1, 1, (256, d_in))
    t = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2])[:, None]
    p = mo.init_params(d_in, width, d_out, 3)
    m = np.zeros(p.size)
    v = np.zeros(p.size)
    l0, _ = mo.loss_and_grad(p, x, t, d_in, width, d_out)
    for step in range(1, 301):
        l, gr = mo.loss_and_grad(p, x, t, d_in, width, d_out)
        p, m, v = mo.adam_step(p, gr, m, v, step, 1e-2)
    l1, _ = mo.loss_and_grad(p, x, t, d_in, width, d_out)
    assert l1 < 0.05 * l0

"""Pins of the warm-start network oracle: the analytic gradient against
central finite differences of the loss (with the BF16 rounding of the weights
frozen at the evaluation point), BF16 rounding against known values, Adam
against its closed forms (the first step, two steps by hand, the bias-corrected
moments as normalised exponential averages) with planted mistakes caught, and
Adam reducing the loss on a fixed regression problem."""
import numpy as np
import pytest

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


# ---- Adam pinned to closed forms (Kingma & Ba, Algorithm 1)

def test_adam_first_step_is_lr_times_sign():
    # zero moments: the bias-corrected first and second moments after one
    # step are g and g^2, so every parameter moves by lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 3e-4, 0.0, -7.25])
    p = np.array([1.0, -1.0, 0.25, 2.0, 0.0], dtype=np.float32)
    lr, eps = 1e-2, 1e-8
    p1, m, v = mo.adam_step(p, g, np.zeros(5), np.zeros(5), 1, lr, eps=eps)
    want = p.astype(np.float64) - lr * g / (np.abs(g) + eps)
    assert np.allclose(p1, want.astype(np.float32), rtol=0, atol=2e-7)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_two_steps_by_hand():
    # g1 = (0.5, -2), g2 = (1, 3), beta1 0.9, beta2 0.999, lr 0.1, eps 0:
    # mhat2 = (0.9 g1 + g2) / 1.9 = (0.7631578947, 0.6315789474)
    # vhat2 = (0.999 g1^2 + g2^2) / 1.999 = (0.6251875938, 6.5012506253)
    # step2 = lr mhat2 / sqrt(vhat2) = (0.0965182, 0.0247702)
    p = np.zeros(2, dtype=np.float32)
    m = np.zeros(2)
    v = np.zeros(2)
    p, m, v = mo.adam_step(p, np.array([0.5, -2.0]), m, v, 1, 0.1, eps=0.0)
    assert np.allclose(p, [-0.1, 0.1], atol=1e-7)
    p2, m, v = mo.adam_step(p, np.array([1.0, 3.0]), m, v, 2, 0.1, eps=0.0)
    assert np.allclose(p2 - p, [-0.0965182, -0.0247702], atol=2e-7)


def test_adam_moments_are_normalised_exponential_averages():
    # bias correction turns the running moments into averages of g and g^2
    # with weights beta^(t-i) normalised to sum 1 (any t, any beta)
    g = np.random.default_rng(5).standard_normal((9, 4))
    b1, b2, lr, eps = 0.8, 0.95, 1e-3, 1e-8
    p = np.zeros(4, dtype=np.float32)
    m = np.zeros(4)
    v = np.zeros(4)
    for t in range(1, 10):
        p0 = p.astype(np.float64)
        p, m, v = mo.adam_step(p, g[t - 1], m, v, t, lr, b1=b1, b2=b2, eps=eps)
        w1 = b1 ** np.arange(t - 1, -1, -1.0)
        w2 = b2 ** np.arange(t - 1, -1, -1.0)
        mh = (w1[:, None] * g[:t]).sum(0) / w1.sum()
        vh = (w2[:, None] * g[:t] ** 2).sum(0) / w2.sum()
        assert np.allclose(p0 - lr * mh / (np.sqrt(vh) + eps), p, rtol=0, atol=1e-7)


@pytest.mark.parametrize("old,new", [
    ("mh = m / (1 - b1**step)", "mh = m"),                       # no bias correction of m
    ("vh = v / (1 - b2**step)", "vh = v"),                       # no bias correction of v
    ("m = b1 * m + (1 - b1) * g", "m = b2 * m + (1 - b2) * g"),  # beta1 and beta2 swapped
    ("v = b2 * v + (1 - b2) * g * g", "v = b1 * v + (1 - b1) * g * g"),
    ("(np.sqrt(vh) + eps)", "(vh + eps)"),                       # missing square root
])
def test_adam_pins_catch_planted_mistakes(old, new):
    import inspect
    import types
    src = inspect.getsource(mo)
    assert src.count(old) == 1
    mod = types.ModuleType("mlp_mutant")
    exec(compile(src.replace(old, new), "<mlp mutant>", "exec"), mod.__dict__)
    saved = mo.adam_step
    caught = 0
    try:
        mo.adam_step = mod.adam_step
        for pin in (test_adam_first_step_is_lr_times_sign, test_adam_two_steps_by_hand,
                    test_adam_moments_are_normalised_exponential_averages):
            try:
                pin()
            except AssertionError:
                caught += 1
    finally:
        mo.adam_step = saved
    assert caught >= 1

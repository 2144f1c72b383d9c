"""Pins of the FP64 surrogate MLP: parameter gradients and the input
gradient against central finite differences; the Adam step against its
closed form on a quadratic; bfloat16 rounding against known bit patterns."""
import numpy as np

from oracle import mlp


def _setup(n=16, seed=0):
    rng = np.random.default_rng(seed)
    th = mlp.init(seed, sigma=3.0).astype(np.float64)
    x = rng.uniform(-5, 5, (n, 3))
    t = rng.uniform(0, 3, n)
    return th, x, t, np.array([0.5, -0.2, 1.0]), 6.0, 2.0


def test_parameter_gradient_fd():
    th, x, t, c, h, s = _setup()
    L, g = mlp.loss_and_grad(th, x, t, c, h, s)
    rng = np.random.default_rng(1)
    idx = rng.choice(np.arange(mlp.NF * 3, mlp.NPARAMS), 60, replace=False)
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(th); e[i] = eps
        fd = (mlp.loss_and_grad(th + e, x, t, c, h, s)[0] - mlp.loss_and_grad(th - e, x, t, c, h, s)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert np.all(g[:mlp.NF * 3] == 0)


def test_input_gradient_fd():
    th, x, t, c, h, s = _setup(8, 2)
    y, dx, _ = mlp.forward(th, x, c, h, s)
    eps = 1e-6
    for j in range(3):
        e = np.zeros(3); e[j] = eps
        fd = (mlp.forward(th, x + e, c, h, s)[0] - mlp.forward(th, x - e, c, h, s)[0]) / (2 * eps)
        assert np.allclose(dx[:, j], fd, atol=1e-7, rtol=1e-6)


def test_adam_closed_form():
    # first step of Adam moves every coordinate by lr * sign(grad)
    th = np.zeros(mlp.NPARAMS)
    g = np.linspace(-1, 1, mlp.NPARAMS)
    g = np.where(np.abs(g) < 0.1, 0.3, g)
    t2, m, v = mlp.adam(th, g, np.zeros_like(g), np.zeros_like(g), 1, 0.01)
    sl = slice(mlp.NF * 3, None)
    assert np.allclose(t2[sl], -0.01 * np.sign(g[sl]), atol=1e-9)
    assert np.all(t2[:mlp.NF * 3] == 0)


def test_round_bf16():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159265, -2.5e-3], np.float32)
    r = mlp.round_bf16(a)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie -> even
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == 3.140625
    assert abs(r[4] + 2.5e-3) <= 2 ** -9 * 2.5e-3 * 2


def test_round_bf16_matches_torch():
    import torch
    a = np.random.default_rng(5).standard_normal(10000).astype(np.float32) * 10.0 ** np.arange(-4, 6).repeat(1000)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.round_bf16(a), ref)


def test_mixed_precision_mode():
    """The stored-precision evaluation is the exact network with every GEMM
    operand perturbed by at most one rounding: it equals the bf16-weight
    evaluation once the activations are representable, and stays within a
    few bfloat16 units of it otherwise."""
    th, x, t, c, h, s = _setup(64, 3)
    y0, d0, _ = mlp.forward(th, x, c, h, s, bf16=True)
    y1, d1, _ = mlp.forward(th, x, c, h, s, mixed=True)
    assert not np.array_equal(y0, y1)
    u = 2.0 ** -8
    assert np.abs(y1 - y0).max() <= 8 * u * s * np.abs(y0).max()
    assert np.abs(d1 - d0).max() <= 16 * u * np.abs(d0).max()
    # zero hidden weights: only b's reach the output, so no rounding matters
    th2 = th.copy()
    o = mlp.NF * 3
    th2[o:] = 0.0
    th2[-1] = 0.75
    ya, _, _ = mlp.forward(th2, x, c, h, s, mixed=True)
    assert np.all(ya == s * 0.75)

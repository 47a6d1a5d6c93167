"""Pins of the FP64 MLP oracle (oracle/mlp.c): closed-form layers, central
finite differences of the loss, and a hand-computed Adam step."""
import numpy as np

import oracle


def _rand(dims, S, seed=0):
    rng = np.random.default_rng(seed)
    n = oracle.mlp_nparams(*dims)
    return rng.normal(0, 0.4, n), rng.normal(0, 1, (S, dims[0])), rng.normal(0, 1, (S, dims[2]))


def test_forward_against_numpy_matrices():
    dims = (7, 11, 5)
    p, x, _ = _rand(dims, 4)
    n_in, n_h, n_out = dims
    o = 0
    W1 = p[o:o + n_h * n_in].reshape(n_h, n_in); o += n_h * n_in
    b1 = p[o:o + n_h]; o += n_h
    W2 = p[o:o + n_h * n_h].reshape(n_h, n_h); o += n_h * n_h
    b2 = p[o:o + n_h]; o += n_h
    W3 = p[o:o + n_out * n_h].reshape(n_out, n_h); o += n_out * n_h
    b3 = p[o:o + n_out]
    h1 = np.maximum(x @ W1.T + b1, 0); h2 = np.maximum(h1 @ W2.T + b2, 0)
    y, g1, g2 = oracle.mlp_forward(dims, p, x)
    np.testing.assert_allclose(y, h2 @ W3.T + b3, atol=1e-13)
    np.testing.assert_allclose(g1, h1, atol=1e-13)


def test_gradient_matches_central_differences():
    dims = (6, 9, 4)
    p, x, t = _rand(dims, 5, seed=3)
    L, g = oracle.mlp_loss_grad(dims, p, x, t)
    rng = np.random.default_rng(1)
    idx = rng.choice(p.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (oracle.mlp_loss_grad(dims, pp, x, t)[0] - oracle.mlp_loss_grad(dims, pm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_loss_of_a_perfect_fit_is_zero_and_gradient_vanishes():
    dims = (3, 4, 2)
    p, x, _ = _rand(dims, 6, seed=5)
    y, _, _ = oracle.mlp_forward(dims, p, x)
    L, g = oracle.mlp_loss_grad(dims, p, x, y)
    assert L < 1e-28 and np.abs(g).max() < 1e-14


def test_adam_first_step_is_sign_times_lr():
    # with m = v = 0, step 1 moves each parameter by -lr * g/(|g| + eps')
    p = np.array([1.0, -2.0, 0.5]); g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3); v = np.zeros(3)
    q = p.copy()
    oracle.adam_step(q, g, m, v, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(q, p - 0.01 * np.sign(g), atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, atol=1e-16)
    np.testing.assert_allclose(v, 0.001 * g * g, atol=1e-16)

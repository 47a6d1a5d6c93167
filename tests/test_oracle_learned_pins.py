"""Pins of the learned preconditioner's oracle (oracle/learned.py), CPU.

The map z = D^-1 r + gamma sum_e G_e^T (w ||r_e|| net([r_e/||r_e||, g_e])) has no
published values; it is pinned by networks whose output is known in closed
form and by its invariants:
  * an identity network (net(x)[:P^3] = x[:P^3], built from ReLU pairs) makes
    the correction at an interior node exactly r_i (the element values are
    rescaled back by ||r_e|| and averaged with weights 1/multiplicity):
    z = D^-1 r + gamma r -- a dropped rescale, a missing average or a wrong
    weight index fails it;
  * a network with zero last-layer weights and bias 1 gives, at each interior
    node, the mean over its elements of ||r_e||;
  * positive homogeneity z(alpha r) = alpha z(r), alpha > 0; gamma = 0 is Jacobi;
  * Cartesian bricks have corner features exactly (+-1/2)^3 and log kappa 0.
"""
import numpy as np

import fem_inputs
import oracle
from oracle import learned


def _mesh(n, p, perturb=0.1, shuffle=None):
    return fem_inputs.box_mesh(n, p, perturb=perturb, seed=3, shuffle_seed=shuffle)


def _identity_net(P3, n_in, n_h, n_out):
    assert n_h >= 2 * P3 and n_out >= P3
    W1 = np.zeros((n_h, n_in)); b1 = np.zeros(n_h)
    W2 = np.eye(n_h); b2 = np.zeros(n_h)
    W3 = np.zeros((n_out, n_h)); b3 = np.zeros(n_out)
    for a in range(P3):
        W1[a, a] = 1.0
        W1[P3 + a, a] = -1.0
        W3[a, a] = 1.0
        W3[a, P3 + a] = -1.0
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def _setup(n=3, p=2, shuffle=5):
    m = _mesh(n, p, shuffle=shuffle)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, p + 2)
    diag = orc.diagonal()
    r = np.random.default_rng(9).uniform(-1, 1, m["N"])
    return m, diag, r


def test_identity_network_gives_jacobi_plus_gamma_r():
    m, diag, r = _setup()
    P3 = (m["p"] + 1) ** 3
    dims = (P3 + 32 + 5, 2 * P3 + 3, P3 + 2)
    params = _identity_net(P3, *dims)
    feat = learned.features(m)
    inner = m["dirichlet"] == 0
    for gamma in (1.0, 0.37):
        z = learned.precond_apply(m, diag, dims, params, r, gamma, feat)
        want = np.where(inner, r / diag + gamma * r, 0.0)
        assert np.max(np.abs(z - want)) <= 1e-13 * np.max(np.abs(want))


def test_bias_network_gives_mean_element_norm():
    m, diag, r = _setup(n=2, p=3)
    P3 = (m["p"] + 1) ** 3
    dims = (P3 + 32, 16, P3)
    n_in, n_h, n_out = dims
    rng = np.random.default_rng(1)
    W1 = rng.normal(size=n_h * n_in); W2 = rng.normal(size=n_h * n_h)
    params = np.concatenate([W1, np.zeros(n_h), W2, np.zeros(n_h), np.zeros(n_out * n_h),
                             np.ones(n_out)])
    z = learned.precond_apply(m, diag, dims, params, r, 1.0, learned.features(m))
    en = m["elem_nodes"]
    sums = np.zeros(m["N"]); cnt = np.zeros(m["N"])
    for e in range(m["E"]):
        nrm = np.linalg.norm(r[en[e]])
        for i in set(en[e].tolist()):
            sums[i] += nrm
            cnt[i] += 1
    inner = m["dirichlet"] == 0
    want = np.where(inner, r / diag + sums / np.maximum(cnt, 1), 0.0)
    assert np.max(np.abs(z - want)) <= 1e-13 * np.max(np.abs(want))


def test_homogeneity_and_gamma_zero():
    m, diag, r = _setup(n=2, p=1)
    P3 = 8
    dims = (64, 32, 32)
    params = fem_inputs.mlp_init(*dims, seed=2, out_scale=1.0).astype(np.float64)
    feat = learned.features(m)
    z1 = learned.precond_apply(m, diag, dims, params, r, 1.0, feat)
    z2 = learned.precond_apply(m, diag, dims, params, 3.7 * r, 1.0, feat)
    assert np.max(np.abs(z2 - 3.7 * z1)) <= 1e-12 * np.max(np.abs(z2))
    z0 = learned.precond_apply(m, diag, dims, params, r, 0.0, feat)
    inner = m["dirichlet"] == 0
    jac = np.where(inner, r / diag, 0.0)
    assert np.max(np.abs(z0 - jac)) <= 1e-15 * np.max(np.abs(jac))
    # the network part is not negligible here (the homogeneity check has teeth)
    assert np.linalg.norm(z1 - z0) > 0.1 * np.linalg.norm(z0)
    assert P3 == (m["p"] + 1) ** 3


def test_cartesian_features():
    m = _mesh(3, 2, perturb=0.0)
    g = learned.features(m)
    for v in range(8):
        sgn = np.array([1 if v & 1 else -1, 1 if v & 2 else -1, 1 if v & 4 else -1]) * 0.5
        assert np.allclose(g[:, 3 * v:3 * v + 3], sgn, atol=1e-14, rtol=0)
    assert not g[:, 24:].any()
    # perturbed elements: the offsets keep zero mean, unit-cube rms scaling
    gp = learned.features(_mesh(3, 2))
    off = gp[:, :24].reshape(-1, 8, 3)
    assert np.allclose(off.sum(axis=1), 0.0, atol=1e-13)
    assert np.allclose(np.sqrt((off ** 2).sum(axis=(1, 2)) / 8.0), np.sqrt(3.0) / 2.0, atol=1e-13)

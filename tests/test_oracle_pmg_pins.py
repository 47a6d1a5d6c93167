"""Pins of the p-multigrid oracle (oracle/pmg.py), CPU only.

Each check ties the oracle to a fact outside itself: the published SplitMix64
outputs, polynomial reproduction of Lagrange interpolation, exact transfer of
linear fields on curved (trilinear) bricks, the Galerkin identity
A_c = P^T A_f P on Cartesian bricks (both sides integrate exactly), the
closed-form Chebyshev error polynomial T_m((theta - lambda)/delta) /
T_m(theta/delta), power iteration on a known spectrum, and the symmetry of a
V-cycle with an exact coarse solve.
"""
import json
import os
import types

import numpy as np
import pytest

import fem_inputs
import oracle
from oracle import pmg

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_matches_published_outputs():
    g = json.load(open(os.path.join(GOLD, "splitmix64_seed0.json")))
    out = pmg.splitmix64(4, g["seed"])
    assert [int(v) for v in out] == [int(h, 16) for h in g["outputs_hex"]]
    v = pmg.start_vector(1000, 0)
    assert np.all(v >= -0.5) and np.all(v < 0.5) and abs(v.mean()) < 0.05


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (4, 8), (3, 7), (5, 5)])
def test_interpolation_reproduces_polynomials(pc, pf):
    I = pmg.interpolation_1d(pc, pf)
    zc, _ = oracle.gauss_lobatto(pc + 1)
    zf, _ = oracle.gauss_lobatto(pf + 1)
    for k in range(pc + 1):
        np.testing.assert_allclose(I @ zc ** k, zf ** k, atol=1e-13)
    np.testing.assert_allclose(I.sum(axis=1), 1.0, atol=1e-14)
    assert I[0, 0] == 1.0 and np.all(I[0, 1:] == 0.0)
    assert I[-1, -1] == 1.0 and np.all(I[-1, :-1] == 0.0)
    if pc == pf:
        np.testing.assert_allclose(I, np.eye(pc + 1), atol=1e-14)


def _levels(n, orders, perturb, seed=3):
    return [pmg.Level(fem_inputs.box_mesh(n, p, perturb=perturb, seed=seed)) for p in orders]


@pytest.mark.parametrize("pf,pc", [(2, 1), (4, 2), (3, 1)])
def test_prolongation_is_exact_on_linear_fields_of_curved_bricks(pf, pc):
    fine, coarse = _levels(3, (pf, pc), perturb=0.15)
    a = np.array([0.3, -1.2, 0.7])
    xc = oracle.nodes_from_vertices(coarse.mesh) @ a + 0.25
    xf = oracle.nodes_from_vertices(fine.mesh) @ a + 0.25
    np.testing.assert_allclose(pmg.prolong(fine, coarse, xc, masked=False), xf, atol=1e-13)


def test_prolongation_is_exact_on_quadratics_of_cartesian_bricks():
    fine, coarse = _levels(2, (4, 2), perturb=0.0)
    f = lambda X: X[:, 0] ** 2 + X[:, 1] * X[:, 2] - 0.5 * X[:, 2] ** 2
    xc = f(oracle.nodes_from_vertices(coarse.mesh))
    xf = f(oracle.nodes_from_vertices(fine.mesh))
    np.testing.assert_allclose(pmg.prolong(fine, coarse, xc, masked=False), xf, atol=1e-13)


def test_restriction_is_the_transpose_of_prolongation():
    fine, coarse = _levels(3, (4, 2), perturb=0.1)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(fine.N)
    v = rng.standard_normal(coarse.N)
    lhs = pmg.restrict(fine, coarse, r) @ v
    rhs = r @ pmg.prolong(fine, coarse, v)
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("pf,pc", [(2, 1), (4, 2)])
def test_galerkin_identity_on_cartesian_bricks(pf, pc):
    # the coarse space is a subspace of the fine one and both rules integrate
    # the (polynomial) integrands exactly on affine bricks
    fine, coarse = _levels(2, (pf, pc), perturb=0.0)
    Af = fine.op.assembled()
    Ac = coarse.op.assembled()
    P = np.stack([pmg.prolong(fine, coarse, e, masked=False) for e in np.eye(coarse.N)], axis=1)
    np.testing.assert_allclose(P.T @ Af @ P, Ac, atol=1e-12 * np.abs(Ac).max())


def _diag_level(lam):
    n = lam.size
    return types.SimpleNamespace(A=lambda v: lam * v, dinv=np.ones(n), diag=np.ones(n),
                                 inner=np.ones(n, dtype=bool), N=n)


def _cheb_T(m, x):
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    big = ~inside
    out[big] = np.sign(x[big]) ** m * np.cosh(m * np.arccosh(np.abs(x[big])))
    return out


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_chebyshev_error_polynomial_is_the_scaled_chebyshev_polynomial(degree):
    lmax = 4.0
    lam = np.concatenate([np.linspace(0.05, 4.4, 41), [0.01, 4.0]])
    lev = _diag_level(lam)
    e = np.ones_like(lam)
    z = pmg.chebyshev(lev, lam * e, lmax, degree, lo=0.1, hi=1.1)
    a, b = 0.1 * lmax, 1.1 * lmax
    theta, delta = (a + b) / 2, (b - a) / 2
    expect = _cheb_T(degree, (theta - lam) / delta) / _cheb_T(degree, np.array([theta / delta]))
    np.testing.assert_allclose(e - z, expect, atol=1e-12)


def test_power_iteration_on_a_known_spectrum():
    lam = np.linspace(1.0, 10.0, 200)
    lev = _diag_level(lam)
    est = pmg.power_lmax(lev, 400)
    assert est <= 10.0 * (1 + 1e-12)
    assert est >= 9.9


def test_vcycle_with_exact_coarse_solve_is_symmetric_positive_definite():
    levels = _levels(2, (4, 2, 1), perturb=0.1)
    lmax = [pmg.power_lmax(l, 30) for l in levels]
    Ac = levels[-1].op.assembled()
    rng = np.random.default_rng(1)
    inner = levels[0].inner
    r = np.where(inner, rng.standard_normal(levels[0].N), 0.0)
    s = np.where(inner, rng.standard_normal(levels[0].N), 0.0)
    Br = pmg.vcycle(levels, lmax, r, coarse_exact=Ac)
    Bs = pmg.vcycle(levels, lmax, s, coarse_exact=Ac)
    assert abs(s @ Br - r @ Bs) <= 1e-12 * abs(s @ Br)
    assert r @ Br > 0 and s @ Bs > 0
    # Dirichlet rows stay zero
    assert np.all(Br[~inner] == 0.0)


def test_fcg_with_jacobi_is_pcg_and_pmg_cuts_iterations():
    levels = _levels(4, (4, 2, 1), perturb=0.1)
    L0 = levels[0]
    b = fem_inputs.rhs_uniform(L0.N, L0.mesh["dirichlet"], seed=4)
    xj, kj, _ = oracle.pcg(L0.op, b, L0.mesh["dirichlet"], rtol=1e-10)
    xf, kf = pmg.fcg(L0, b, lambda r: L0.dinv * r, rtol=1e-10)
    assert abs(kf - kj) <= 1
    assert np.linalg.norm(xf - xj) <= 1e-8 * np.linalg.norm(xj)
    lmax = [pmg.power_lmax(l, 20) for l in levels]
    xm, km = pmg.fcg(L0, b, lambda r: pmg.vcycle(levels, lmax, r, coarse_its=20), rtol=1e-10)
    res = np.where(L0.inner, b - L0.op.apply(xm), 0.0)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(np.where(L0.inner, b, 0.0))
    assert km * 4 <= kj

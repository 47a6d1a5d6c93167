"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test compares the oracle with something other than itself: closed-form
quadrature rules, numpy's independent routines, exact polynomial integration,
integral identities of the bilinear forms, convergence orders, dense linear
algebra on tiny meshes.  Operators and problems: section "Benchmarks" (BP1-BP6,
A_ij and B_ij, Gauss-Legendre q=p+2 / Gauss-Lobatto q=p+1, CG).
"""
import json
import math
import os

import numpy as np
import numpy.polynomial.legendre as npleg
import numpy.polynomial.polynomial as nppoly
import pytest

import fem_inputs
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ev(s):
    return eval(s, {"sqrt": math.sqrt})


# ---------------------------------------------------------------- quadrature

@pytest.mark.parametrize("q", ["1", "2", "3", "4"])
def test_gauss_legendre_closed_forms(q):
    g = json.load(open(os.path.join(GOLD, "quadrature_closed_forms.json")))["gauss_legendre"][q]
    x, w = oracle.gauss_legendre(int(q))
    np.testing.assert_allclose(x, [_ev(s) for s in g["x"]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [_ev(s) for s in g["w"]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("P", ["2", "3", "4", "5"])
def test_gauss_lobatto_closed_forms(P):
    g = json.load(open(os.path.join(GOLD, "quadrature_closed_forms.json")))["gauss_lobatto"][P]
    x, w = oracle.gauss_lobatto(int(P))
    np.testing.assert_allclose(x, [_ev(s) for s in g["x"]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [_ev(s) for s in g["w"]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("q", range(1, 13))
def test_gauss_legendre_matches_numpy_and_is_exact(q):
    x, w = oracle.gauss_legendre(q)
    xr, wr = npleg.leggauss(q)
    np.testing.assert_allclose(x, xr, atol=2e-15)
    np.testing.assert_allclose(w, wr, atol=2e-15)
    for k in range(2 * q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 2e-14
    # degree 2q is not integrated exactly
    assert abs(np.sum(w * x ** (2 * q)) - 2.0 / (2 * q + 1)) > 1e-11


@pytest.mark.parametrize("P", range(2, 12))
def test_gauss_lobatto_matches_numpy_roots_and_is_exact(P):
    p = P - 1
    x, w = oracle.gauss_lobatto(P)
    inner = np.sort(npleg.Legendre.basis(p).deriv().roots().real) if p > 1 else np.array([])
    np.testing.assert_allclose(x, np.concatenate([[-1.0], inner, [1.0]]), atol=1e-14)
    for k in range(2 * P - 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 2e-14
    assert abs(np.sum(w) - 2.0) < 1e-14


# ---------------------------------------------------------------- 1D basis

def _numpy_lagrange(p):
    """Lagrange polynomials on the Gauss-Lobatto nodes built with numpy only."""
    inner = np.sort(npleg.Legendre.basis(p).deriv().roots().real) if p > 1 else np.array([])
    z = np.concatenate([[-1.0], inner, [1.0]])
    polys = []
    for a in range(p + 1):
        others = np.delete(z, a)
        c = nppoly.polyfromroots(others)
        polys.append(c / nppoly.polyval(z[a], c))
    return z, polys


@pytest.mark.parametrize("p", range(1, 9))
def test_lagrange_basis_identities(p):
    z, polys = _numpy_lagrange(p)
    r = np.linspace(-1, 1, 17)
    v, d = oracle.lagrange_1d(p, r)
    # against numpy's polynomial construction
    for a, c in enumerate(polys):
        np.testing.assert_allclose(v[:, a], nppoly.polyval(r, c), atol=1e-12)
        np.testing.assert_allclose(d[:, a], nppoly.polyval(r, nppoly.polyder(c)), atol=1e-10)
    vz, dz = oracle.lagrange_1d(p, z)
    np.testing.assert_allclose(vz, np.eye(p + 1), atol=1e-14)       # l_a(z_b) = delta
    np.testing.assert_allclose(v.sum(1), 1.0, atol=1e-13)             # partition of unity
    np.testing.assert_allclose(d.sum(1), 0.0, atol=1e-11)             # rows of D sum to 0
    for k in range(1, p + 1):                                         # exact derivative
        np.testing.assert_allclose(d @ (z ** k), k * r ** (k - 1), atol=1e-11)


# ---------------------------------------------------------------- mesh

def test_nodes_of_unperturbed_mesh_are_the_lattice():
    n, p = 3, 4
    m = fem_inputs.box_mesh(n, p, perturb=0.0)
    xyz = oracle.nodes_from_vertices(m)
    z, _ = oracle.gauss_lobatto(p + 1)
    one = np.concatenate([e / n + (z[:-1] + 1) / (2 * n) for e in range(n)] + [[1.0]])
    M = m["M"]
    I = np.arange(m["N"]) % M
    J = (np.arange(m["N"]) // M) % M
    K = np.arange(m["N"]) // (M * M)
    np.testing.assert_allclose(xyz[:, 0], one[I], atol=1e-15)
    np.testing.assert_allclose(xyz[:, 1], one[J], atol=1e-15)
    np.testing.assert_allclose(xyz[:, 2], one[K], atol=1e-15)


# ---------------------------------------------------------------- operators

def _op(n, p, kind, quad, q=None, perturb=0.1, seed=3, ncomp=1, **kw):
    m = fem_inputs.box_mesh(n, p, perturb=perturb, seed=seed)
    if q is None:
        q = p + 2 if quad == oracle.GAUSS else p + 1
    return m, oracle.Operator(m, kind, quad, q, ncomp=ncomp, **kw)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_of_one_is_the_volume_gauss(p):
    m, op = _op(3, p, oracle.MASS, oracle.GAUSS)
    one = np.ones(m["N"])
    assert abs(one @ op.apply(one) - 1.0) < 1e-13


@pytest.mark.parametrize("p", [2, 3, 5])
def test_mass_of_one_is_the_volume_lobatto(p):
    # det J of a trilinear map has degree <= 2 per direction: GLL with p+1 >= 3
    # points integrates it exactly.
    m, op = _op(3, p, oracle.MASS, oracle.LOBATTO)
    one = np.ones(m["N"])
    assert abs(one @ op.apply(one) - 1.0) < 1e-13


def test_mass_lobatto_p1_is_not_exact():
    m, op = _op(3, 1, oracle.MASS, oracle.LOBATTO, perturb=0.1)
    one = np.ones(m["N"])
    assert abs(one @ op.apply(one) - 1.0) > 1e-8


@pytest.mark.parametrize("quad,p", [(oracle.GAUSS, 1), (oracle.GAUSS, 3), (oracle.LOBATTO, 3),
                                    (oracle.LOBATTO, 6)])
def test_diffusion_annihilates_constants(quad, p):
    m, op = _op(2, p, oracle.DIFFUSION, quad)
    y = op.apply(np.ones(m["N"]))
    assert np.abs(y).max() < 1e-12


@pytest.mark.parametrize("quad,p", [(oracle.GAUSS, 1), (oracle.GAUSS, 2), (oracle.GAUSS, 4),
                                    (oracle.LOBATTO, 3), (oracle.LOBATTO, 5)])
def test_diffusion_exact_on_linear_fields(quad, p):
    m, op = _op(2, p, oracle.DIFFUSION, quad)
    xyz = op.node_xyz
    a = np.array([1.0, -2.0, 0.5]); b = np.array([0.3, 1.5, -2.5])
    u, v = xyz @ a, xyz @ b
    Au = op.apply(u)
    assert abs(v @ Au - a @ b) < 1e-12                     # (a.b) * volume
    interior = m["dirichlet"] == 0
    assert np.abs(Au[interior]).max() < 1e-12              # int grad phi_i . a = 0


@pytest.mark.parametrize("kind", [oracle.MASS, oracle.DIFFUSION])
@pytest.mark.parametrize("quad,p", [(oracle.GAUSS, 2), (oracle.LOBATTO, 4)])
def test_symmetry(kind, quad, p):
    m, op = _op(2, p, kind, quad)
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-1, 1, (2, m["N"]))
    a, b = y @ op.apply(x), x @ op.apply(y)
    assert abs(a - b) <= 1e-14 * max(abs(a), 1.0) * 10


def _exact_1d(p, h, quad):
    """1D mass and stiffness on an interval of length h by exact polynomial
    integration (numpy), plus the diagonal Gauss-Lobatto mass."""
    z, polys = _numpy_lagrange(p)
    P = p + 1
    Mx = np.zeros((P, P)); Kx = np.zeros((P, P))
    for a in range(P):
        for b in range(P):
            mi = nppoly.polyint(nppoly.polymul(polys[a], polys[b]))
            ki = nppoly.polyint(nppoly.polymul(nppoly.polyder(polys[a]), nppoly.polyder(polys[b])))
            Mx[a, b] = (nppoly.polyval(1, mi) - nppoly.polyval(-1, mi)) * h / 2
            Kx[a, b] = (nppoly.polyval(1, ki) - nppoly.polyval(-1, ki)) * 2 / h
    return Mx, Kx


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_cartesian_element_is_kronecker_sum_gauss(p):
    m, opK = _op(1, p, oracle.DIFFUSION, oracle.GAUSS, perturb=0.0)
    _, opM = _op(1, p, oracle.MASS, oracle.GAUSS, perturb=0.0)
    Mx, Kx = _exact_1d(p, 1.0, oracle.GAUSS)
    K3 = np.kron(Mx, np.kron(Mx, Kx)) + np.kron(Mx, np.kron(Kx, Mx)) + np.kron(Kx, np.kron(Mx, Mx))
    M3 = np.kron(Mx, np.kron(Mx, Mx))
    np.testing.assert_allclose(opK.element_matrix(0), K3, atol=1e-12)
    np.testing.assert_allclose(opM.element_matrix(0), M3, atol=1e-14)
    if p == 1:  # textbook 1D matrices, h = 1
        np.testing.assert_allclose(Mx, np.array([[2, 1], [1, 2]]) / 6, atol=1e-15)
        np.testing.assert_allclose(Kx, np.array([[1, -1], [-1, 1]]), atol=1e-15)


@pytest.mark.parametrize("p", [2, 4, 7])
def test_cartesian_element_lobatto(p):
    # GLL stiffness integrand has degree 2p-2 <= 2(p+1)-3: exact; GLL mass is the
    # diagonal (lumped) tensor of the weights.
    h = 0.5
    m = fem_inputs.box_mesh(2, p, perturb=0.0)
    opK = oracle.Operator(m, oracle.DIFFUSION, oracle.LOBATTO, p + 1)
    opM = oracle.Operator(m, oracle.MASS, oracle.LOBATTO, p + 1)
    Mx, Kx = _exact_1d(p, h, oracle.LOBATTO)
    K3 = np.kron(Mx, np.kron(Mx, Kx)) + np.kron(Mx, np.kron(Kx, Mx)) + np.kron(Kx, np.kron(Mx, Mx))
    # the GLL mass inside the stiffness sum is the lumped one
    inner = np.sort(npleg.Legendre.basis(p).deriv().roots().real)
    z = np.concatenate([[-1.0], inner, [1.0]])
    wl = 2.0 / (p * (p + 1) * npleg.legval(z, [0] * p + [1]) ** 2)
    Ml = np.diag(wl * h / 2)
    K3l = np.kron(Ml, np.kron(Ml, Kx)) + np.kron(Ml, np.kron(Kx, Ml)) + np.kron(Kx, np.kron(Ml, Ml))
    for e in range(m["E"]):
        np.testing.assert_allclose(opK.element_matrix(e), K3l, atol=1e-12)
        np.testing.assert_allclose(opM.element_matrix(e), np.kron(Ml, np.kron(Ml, Ml)), atol=1e-15)
    assert np.abs(K3l - K3).max() > 1e-6  # the lumped form differs from the exact one


def test_qdata_of_cartesian_element():
    n, p = 2, 3
    h = 1.0 / n
    m = fem_inputs.box_mesh(n, p, perturb=0.0)
    q = p + 2
    opD = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, q)
    opM = oracle.Operator(m, oracle.MASS, oracle.GAUSS, q)
    xg, wg = npleg.leggauss(q)
    W = np.einsum("k,j,i->kji", wg, wg, wg).ravel()
    for e in range(m["E"]):
        D = opD.qdata(e)
        np.testing.assert_allclose(D[0], W * h / 2, atol=1e-15)
        np.testing.assert_allclose(D[1], W * h / 2, atol=1e-15)
        np.testing.assert_allclose(D[2], W * h / 2, atol=1e-15)
        np.testing.assert_allclose(D[3:], 0.0, atol=1e-15)
        np.testing.assert_allclose(opM.qdata(e)[0], W * (h / 2) ** 3, atol=1e-16)


def test_qdata_of_a_sheared_affine_element():
    # One element with vertices x = F r' + c (r' in [0,1]^3): J = F/2 everywhere,
    # D = w det(J) J^{-1} J^{-T}.
    F = np.array([[1.0, 0.2, 0.1], [0.0, 0.8, -0.3], [0.1, 0.0, 1.2]])
    m = fem_inputs.box_mesh(1, 2, perturb=0.0)
    m["vert_xyz"] = m["vert_xyz"] @ F.T + np.array([0.1, -0.2, 0.3])
    op = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 4)
    J = F / 2
    G = np.linalg.det(J) * np.linalg.inv(J) @ np.linalg.inv(J).T
    xg, wg = npleg.leggauss(4)
    W = np.einsum("k,j,i->kji", wg, wg, wg).ravel()
    D = op.qdata(0)
    for c, (i, k) in enumerate([(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]):
        np.testing.assert_allclose(D[c], W * G[i, k], rtol=1e-13, atol=1e-16)


def test_apply_equals_sum_of_element_matrices_and_diagonal():
    m, op = _op(2, 2, oracle.DIFFUSION, oracle.GAUSS)
    A = op.assembled()
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, m["N"])
    np.testing.assert_allclose(op.apply(x), A @ x, atol=1e-13)
    d = op.diagonal()
    np.testing.assert_allclose(d, np.diag(A), atol=1e-14)
    # brute force: diag_i = (A e_i)_i
    for i in [0, 7, 62, m["N"] - 1]:
        e = np.zeros(m["N"]); e[i] = 1.0
        assert abs(op.apply(e)[i] - d[i]) < 1e-14


def test_apply_subset_and_rows():
    m, op = _op(3, 2, oracle.DIFFUSION, oracle.GAUSS)
    x = np.random.default_rng(2).uniform(-1, 1, m["N"])
    full = op.apply(x)
    parts = op.apply(x, elems=np.arange(0, m["E"], 2)) + op.apply(x, elems=np.arange(1, m["E"], 2))
    np.testing.assert_allclose(parts, full, atol=1e-13)
    rows = np.array([0, 5, 100, 171, m["N"] - 1])
    ptr, el = fem_inputs.elements_of_nodes(m, rows)
    np.testing.assert_allclose(op.apply_rows(x, rows, ptr, el), full[rows], atol=1e-13)


def test_vector_operator_is_componentwise():
    m, op1 = _op(2, 3, oracle.DIFFUSION, oracle.LOBATTO)
    op3 = oracle.Operator(m, oracle.DIFFUSION, oracle.LOBATTO, 4, ncomp=3)
    x = np.random.default_rng(1).uniform(-1, 1, 3 * m["N"])
    y = op3.apply(x).reshape(3, -1)
    for c in range(3):
        np.testing.assert_allclose(y[c], op1.apply(x.reshape(3, -1)[c]), atol=1e-14)


def test_rhs_integrates_the_load():
    # sum_i b_i = int f dV = (2/pi)^3 for f = sin sin sin (partition of unity)
    m, op = _op(4, 3, oracle.MASS, oracle.GAUSS)
    b = op.rhs(0)
    assert abs(b.sum() - (2 / np.pi) ** 3) < 1e-7
    assert abs(op.rhs(1).sum() - 3 * np.pi ** 2 * (2 / np.pi) ** 3) < 1e-5


def test_kappa_random_features_covariance():
    # log kappa = sigma sqrt(2/M) sum cos(w.x+b) has, over the draws of (w,b),
    # mean 0 and covariance sigma^2 exp(-|x-y|^2 / (2 ell^2)) (Rahimi & Recht).
    m = fem_inputs.box_mesh(1, 1, perturb=0.0)
    ell = 0.1
    x0 = np.array([0.3, 0.4, 0.5])
    shifts = [0.0, 0.1, 0.2]
    R = 300
    samples = np.zeros((R, len(shifts) + 1))
    for s in range(R):
        op = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 2,
                             rff=fem_inputs.rff_params(256, ell, seed=s), sigma=1.0)
        samples[s, 0] = np.log(op.kappa(x0))
        for t, d in enumerate(shifts):
            samples[s, t + 1] = np.log(op.kappa(x0 + np.array([d, 0, 0])))
    assert abs(samples[:, 0].mean()) < 0.2
    for t, d in enumerate(shifts):
        cov = np.mean(samples[:, 0] * samples[:, t + 1])
        assert abs(cov - np.exp(-d * d / (2 * ell * ell))) < 0.2


# ---------------------------------------------------------------- solves

def test_tiny_constrained_system_is_spd_and_cg_matches_dense_solve():
    m, op = _op(2, 3, oracle.DIFFUSION, oracle.GAUSS)
    A = op.assembled()
    inner = m["dirichlet"] == 0
    Aii = A[np.ix_(inner, inner)]
    assert np.linalg.eigvalsh(Aii).min() > 0
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=4)
    x, it, hist = oracle.pcg(op, b, m["dirichlet"], rtol=1e-12)
    xd = np.zeros(m["N"])
    xd[inner] = np.linalg.solve(Aii, b[inner])
    cond = np.linalg.cond(Aii)
    assert np.linalg.norm(x - xd) <= 1e-12 * cond * np.linalg.norm(xd)
    assert hist[-1] <= 1e-12 and it < 200
    # Jacobi preconditioning does not lose against plain CG here
    _, it0, _ = oracle.pcg(op, b, m["dirichlet"], rtol=1e-12, precond="none")
    assert it <= it0 + 2


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_bp3_manufactured_convergence_orders(p):
    # L2 error O(h^{p+1}), H1 error O(h^p) on perturbed meshes n = 4, 8 (n = 2
    # is pre-asymptotic); at p = 3, 4 a wrong high-order node, weight or basis
    # derivative drops the slopes (measured 4.05 / 3.05 and 4.86 / 3.88)
    errs = []
    hs = []
    for n in (2, 4, 8):
        m, op = _op(n, p, oracle.DIFFUSION, oracle.GAUSS, seed=11)
        b = op.rhs(1)
        b[m["dirichlet"] == 1] = 0.0
        x, it, hist = oracle.pcg(op, b, m["dirichlet"], rtol=1e-12)
        errs.append(op.error_norms(x))
        hs.append(1.0 / n)
    errs = np.array(errs)
    sl2 = np.polyfit(np.log(hs[1:]), np.log(errs[1:, 0]), 1)[0]
    sh1 = np.polyfit(np.log(hs[1:]), np.log(errs[1:, 1]), 1)[0]
    assert sl2 >= p + 1 - 0.3, sl2
    assert sh1 >= p - 0.3, sh1


def test_bp1_cg_hundred_iterations_projects_the_load():
    # BP1: 100 unpreconditioned CG iterations on B u = b, b_i = int phi_i f:
    # u approaches the L2 projection of f = sin sin sin (error O(h^{p+1})).
    m, op = _op(4, 2, oracle.MASS, oracle.GAUSS, seed=1)
    b = op.rhs(0)
    b[m["dirichlet"] == 1] = 0.0
    x, it, hist = oracle.pcg(op, b, m["dirichlet"], rtol=0.0, maxit=100, precond="none")
    assert it == 100
    l2, _ = op.error_norms(x)
    assert l2 < 5e-3
    assert hist[-1] < 1e-8

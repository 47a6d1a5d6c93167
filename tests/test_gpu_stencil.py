"""The assembled 27-point stencil of p = 1 Gauss diffusion (launch choice 24).

On a lattice mesh (lexicographic n x n x n brick) the FP64 operator's default
p = 1 body is the globally assembled operator, applied row by row in
double-word arithmetic.  It must meet the FP64 bar against the oracle (1e-12
relative l2, random and smooth inputs, even and odd n, the one-element mesh),
give the element-matrix body's result, be deterministic (no atomics), fall
back to the element-matrix body for element lists, be refused on a mesh that
is not a lattice, and carry CG as the oracle's PCG does.
"""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu

STENCIL, ELMAT = 24, 11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def make(n, seed=3, shuffle=None):
    m = fem_inputs.box_mesh(n, 1, perturb=0.1, seed=seed, shuffle_seed=shuffle)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, fem.DIFFUSION, fem.GAUSS, 3)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 3)
    return m, gm, op, orc


def fields(m, seed=0):
    rng = np.random.default_rng(seed)
    M = m["M"]
    g = np.arange(m["N"])
    I, J, K = g % M, (g // M) % M, g // (M * M)
    t = np.pi / max(M - 1, 1)
    out = [rng.uniform(-1, 1, m["N"])]
    if M > 3:   # (on coarser lattices the sine vanishes at every node)
        out.append(np.sin(t * I) * np.sin(2 * t * J) * np.cos(t * K))
    return out


@pytest.mark.parametrize("n", [1, 2, 5, 8, 11])
def test_stencil_matches_oracle_and_element_matrices(n):
    m, gm, op, orc = make(n, seed=10 + n)
    for xv in fields(m, seed=n):
        ref = orc.apply(xv)
        x = torch.from_numpy(xv).cuda()
        y_def = op.apply(x)                 # the default: the stencil
        op.set_launch_shape(fem.F64, STENCIL)
        y24 = op.apply(x)
        y24b = op.apply(x)
        op.set_launch_shape(fem.F64, ELMAT)
        y11 = op.apply(x)
        op.set_launch_shape(fem.F64, STENCIL)
        # deterministic: one thread writes each row, no atomics
        assert torch.equal(y24, y24b) and torch.equal(y_def, y24)
        assert rel(y24.cpu().numpy(), ref) <= 1e-12
        assert rel(y24.cpu().numpy(), y11.cpu().numpy()) <= 1e-13


def test_stencil_refused_on_shuffled_mesh():
    m, gm, op, orc = make(4, shuffle=5)
    with pytest.raises(fem.FemError):
        op.set_launch_shape(fem.F64, STENCIL)
    # the default stays a body that holds any element order
    xv = fields(m)[0]
    assert rel(op.apply(torch.from_numpy(xv).cuda()).cpu().numpy(), orc.apply(xv)) <= 1e-12


def test_stencil_element_list_falls_back():
    m, gm, op, orc = make(6, seed=2)
    op.set_launch_shape(fem.F64, STENCIL)
    rng = np.random.default_rng(4)
    sel = np.sort(rng.choice(m["E"], m["E"] // 3, replace=False)).astype(np.int32)
    xv = rng.uniform(-1, 1, m["N"])
    y = op.apply_elements(torch.from_numpy(sel).cuda(), torch.from_numpy(xv).cuda())
    assert rel(y.cpu().numpy(), orc.apply(xv, elems=sel)) <= 1e-12


@pytest.mark.parametrize("use_graph", [True, False])
def test_stencil_cg_matches_oracle_pcg(use_graph):
    m, gm, op, orc = make(9, seed=6)
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=2)
    xr, itr, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=1e-10)
    x = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
    st = op.cg(torch.from_numpy(b).cuda(), x, precond=fem.PC_JACOBI, rtol=1e-10, use_graph=use_graph)
    assert st["status"] == "FEM_OK"
    assert abs(st["iterations"] - itr) <= 2
    assert rel(x.cpu().numpy(), xr) <= 1e-8
    inner = m["dirichlet"] == 0
    res = np.where(inner, b - orc.apply(x.cpu().numpy()), 0.0)
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(b)


def make32(n, seed=3):
    m = fem_inputs.box_mesh(n, 1, perturb=0.1, seed=seed)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, fem.DIFFUSION, fem.GAUSS, 3, prec=fem.F32)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 3)
    return m, gm, op, orc


@pytest.mark.parametrize("n", [2, 7, 12])
def test_stencil_f32_matches_oracle_and_element_matrices(n):
    # the FP32 stencil: the FP32 bar (1e-5), its own default, deterministic
    m, gm, op, orc = make32(n, seed=20 + n)
    for xv in fields(m, seed=n):
        ref = orc.apply(xv)
        x = torch.from_numpy(xv).cuda().float()
        y_def = op.apply_f32(x)
        op.set_launch_shape(fem.F32, STENCIL)
        y24 = op.apply_f32(x)
        y24b = op.apply_f32(x)
        op.set_launch_shape(fem.F32, 7)
        y7 = op.apply_f32(x)
        op.set_launch_shape(fem.F32, STENCIL)
        assert torch.equal(y24, y24b) and torch.equal(y_def, y24)
        assert rel(y24.double().cpu().numpy(), ref) <= 1e-5
        assert rel(y24.double().cpu().numpy(), y7.double().cpu().numpy()) <= 1e-5
    # the FP64 apply of the same operator keeps its own (double-word) stencil
    xv = fields(m, seed=1)[0]
    assert rel(op.apply(torch.from_numpy(xv).cuda()).cpu().numpy(), orc.apply(xv)) <= 1e-12


def test_stencil_f32_refused_on_fp64_operator():
    m, gm, op, orc = make(3)
    with pytest.raises(fem.FemError):
        op.set_launch_shape(fem.F32, STENCIL)


def test_stencil_refined_solve():
    # FP32 inner CG on the FP32 stencil, FP64 residuals on the double-word one
    m, gm, op, orc = make32(9, seed=8)
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=5)
    x = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
    st = op.solve_refined(torch.from_numpy(b).cuda(), x, rtol=1e-10, inner_rtol=0.1)
    assert st["status"] == "FEM_OK"
    inner = m["dirichlet"] == 0
    res = np.where(inner, b - orc.apply(x.cpu().numpy()), 0.0)
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(b)

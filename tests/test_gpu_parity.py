"""GPU parity: the CUDA operator against the FP64 oracle, element by element,
on seeded perturbed brick meshes spanning several blocks and a ragged tail.

Bar (FP64): relative l2 error <= 1e-12 for the apply and the diagonal,
<= 1e-13 for the geometric data (a handful of FP64 operations per entry).
"""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    fem.lib()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make(name, n, p, seed=5, shuffle=None, prec=fem.F64, rff=None):
    kind, ncomp, quad, dq = fem.BAKE_OFF[name]
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=seed, shuffle_seed=shuffle)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, kind, quad, p + dq, ncomp=ncomp, prec=prec, rff=rff)
    orc = oracle.Operator(m, kind, quad, p + dq, ncomp=ncomp, rff=rff)
    return m, gm, op, orc


def inputs(m, ncomp, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, ncomp * m["N"])
    # a smooth field on the node lattice (index arithmetic only)
    M = m["M"]
    g = np.arange(m["N"])
    I, J, K = g % M, (g // M) % M, g // (M * M)
    t = np.pi / max(M - 1, 1)
    s = np.sin(t * I) * np.sin(2 * t * J) * np.cos(t * K)
    return [x, np.tile(s, ncomp)]


CASES = ([("BP3", p) for p in range(1, 9)] + [("BP5", p) for p in range(1, 9)] +
         [("BP1", p) for p in (1, 2, 4, 8)] + [("BP2", 3), ("BP4", 2), ("BP6", 7), ("BP6", 2)])


@pytest.mark.parametrize("name,p", CASES)
def test_apply_matches_oracle(name, p):
    n = {1: 5, 2: 4, 3: 3, 4: 3, 5: 3, 6: 2, 7: 2, 8: 2}[p]
    m, gm, op, orc = make(name, n, p, shuffle=17)
    for x in inputs(m, op.ncomp):
        y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert rel(y, orc.apply(x)) <= TOL64


@pytest.mark.parametrize("name,p", [("BP3", 3), ("BP5", 7), ("BP1", 2)])
def test_qdata_matches_oracle(name, p):
    m, gm, op, orc = make(name, 2, p)
    for e in range(m["E"]):
        assert rel(op.qdata(e), orc.qdata(e)) <= 1e-13


@pytest.mark.parametrize("name,p", [("BP3", 1), ("BP3", 4), ("BP3", 8), ("BP5", 3), ("BP5", 7),
                                    ("BP1", 2), ("BP6", 4)])
def test_diagonal_matches_oracle(name, p):
    m, gm, op, orc = make(name, 2, p)
    d = op.diagonal().cpu().numpy()
    assert rel(d, orc.diagonal()) <= TOL64


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("p", [1, 3, 6])
def test_rhs_matches_oracle(which, p):
    m, gm, op, orc = make("BP3", 3, p)
    b = op.rhs(which).cpu().numpy()
    assert rel(b, orc.rhs(which)) <= TOL64


def test_apply_elements_subset_and_empty():
    m, gm, op, orc = make("BP3", 4, 3, shuffle=3)
    x = inputs(m, 1)[0]
    sel = np.random.default_rng(1).choice(m["E"], size=23, replace=False).astype(np.int32)
    y = op.apply_elements(torch.from_numpy(sel).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, orc.apply(x, elems=sel)) <= TOL64
    y0 = op.apply_elements(torch.zeros(0, dtype=torch.int32, device="cuda"),
                           torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(y0 == 0.0)


def test_single_element_and_largest_order():
    for name in ("BP3", "BP5", "BP1"):
        m, gm, op, orc = make(name, 1, 8)
        x = inputs(m, 1)[0]
        assert rel(op.apply(torch.from_numpy(x).cuda()).cpu().numpy(), orc.apply(x)) <= TOL64


def test_variable_coefficient_matches_oracle():
    rff = fem_inputs.rff_params(64, 0.1, seed=3)
    m, gm, op, orc = make("BP3", 3, 4, rff=rff)
    for e in (0, 13, 26):
        assert rel(op.qdata(e), orc.qdata(e)) <= 1e-12
    x = inputs(m, 1)[0]
    assert rel(op.apply(torch.from_numpy(x).cuda()).cpu().numpy(), orc.apply(x)) <= TOL64


def test_linear_fields_and_constants():
    # facts that hold at any size: A 1 = 0 and v^T A u = (a.b) vol
    m, gm, op, orc = make("BP3", 6, 3)
    xyz = gm.node_xyz
    one = torch.ones(m["N"], dtype=torch.float64, device="cuda")
    assert op.apply(one).abs().max().item() < 1e-12
    a = np.array([1.0, -2.0, 0.5]); b = np.array([0.3, 1.5, -2.5])
    u = torch.from_numpy(xyz @ a).cuda(); v = torch.from_numpy(xyz @ b).cuda()
    assert abs(torch.dot(v, op.apply(u)).item() - a @ b) < 1e-11


# ---------------------------------------------------------------- solves

@pytest.mark.parametrize("use_graph", [True, False])
def test_cg_jacobi_matches_oracle_pcg(use_graph):
    m, gm, op, orc = make("BP3", 4, 3)
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=2)
    xr, itr, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=1e-10)
    x = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
    st = op.cg(torch.from_numpy(b).cuda(), x, precond=fem.PC_JACOBI, rtol=1e-10,
               use_graph=use_graph)
    assert st["status"] == "FEM_OK"
    assert abs(st["iterations"] - itr) <= 2
    assert rel(x.cpu().numpy(), xr) <= 1e-8
    # true residual of the GPU solution, measured by the oracle
    inner = m["dirichlet"] == 0
    res = np.where(inner, b - orc.apply(x.cpu().numpy()), 0.0)
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(b)


def test_cg_bp1_hundred_iterations_and_graph_replay():
    m, gm, op, orc = make("BP1", 8, 2, seed=1)
    b = orc.rhs(0)
    b[m["dirichlet"] == 1] = 0.0
    xr, itr, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=0.0, maxit=100, precond="none")
    bt = torch.from_numpy(b).cuda()
    for _ in range(2):  # second call replays the captured graph
        x = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
        st = op.cg(bt, x, precond=fem.PC_NONE, maxit=100, rtol=0.0)
        assert st["iterations"] == 100 and st["status"] == "FEM_OK"
        assert rel(x.cpu().numpy(), xr) <= 1e-9


def test_cg_vector_bp6_and_edge_cases():
    m, gm, op, orc = make("BP6", 3, 3)
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=8, ncomp=3)
    xr, itr, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=1e-10)
    x = torch.zeros(3 * m["N"], dtype=torch.float64, device="cuda")
    st = op.cg(torch.from_numpy(b).cuda(), x, rtol=1e-10)
    assert abs(st["iterations"] - itr) <= 2 and rel(x.cpu().numpy(), xr) <= 1e-8
    # b = 0: zero iterations, x = 0 on the interior
    z = torch.zeros_like(x)
    x2 = torch.ones_like(x)
    st = op.cg(z, x2, rtol=1e-10)
    assert st["iterations"] == 0
    # iteration cap -> FEM_ENOCONV
    x3 = torch.zeros_like(x)
    st = op.cg(torch.from_numpy(b).cuda(), x3, rtol=1e-14, maxit=3)
    assert st["status"] == "FEM_ENOCONV" and st["iterations"] == 3


def test_cg_restart_from_iterate_continues_the_solve():
    m, gm, op, orc = make("BP3", 4, 2)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=3)).cuda()
    x = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
    st1 = op.cg(b, x, rtol=1e-4)
    st2 = op.cg(b, x, rtol=1e-10)   # resume from the saved iterate
    assert st2["rnorm"] <= 1e-10 * st2["bnorm"] * 1.0000001
    xr, _, _ = oracle.pcg(orc, b.cpu().numpy(), m["dirichlet"], rtol=1e-12)
    assert rel(x.cpu().numpy(), xr) <= 1e-8


# ---------------------------------------------------------------- trilinear body

@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("ncomp", [1, 3])
def test_trilinear_body_matches_oracle(q, ncomp):
    # p = 1 Gauss diffusion, thread-per-element body (launch choice 6): 9^3
    # elements = 6 blocks of 128 threads with a ragged tail, shuffled order
    m = fem_inputs.box_mesh(9, 1, perturb=0.1, seed=12, shuffle_seed=4)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, fem.DIFFUSION, fem.GAUSS, q, ncomp=ncomp, prec=fem.F32)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, q, ncomp=ncomp)
    for prec, tol in ((fem.F64, TOL64), (fem.F32, 1e-5)):
        for bps in (1, 0):
            op.set_launch_shape(prec, 6, bps)
            for x in inputs(m, ncomp, seed=q):
                xt = torch.from_numpy(x).cuda()
                if prec == fem.F64:
                    y = op.apply(xt).cpu().numpy()
                else:
                    y = op.apply_f32(xt.float()).double().cpu().numpy()
                assert rel(y, orc.apply(x)) <= tol, (prec, bps)
    # a listed subset of elements, and the empty list
    op.set_launch_shape(fem.F64, 6, 0)
    x = inputs(m, ncomp)[0]
    sel = np.random.default_rng(2).choice(m["E"], size=300, replace=False).astype(np.int32)
    y = op.apply_elements(torch.from_numpy(sel).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, orc.apply(x, elems=sel)) <= TOL64
    y0 = op.apply_elements(torch.zeros(0, dtype=torch.int32, device="cuda"),
                           torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(y0 == 0.0)


def test_trilinear_body_in_cg_and_only_where_valid():
    # the fused p^T A p of the trilinear body drives CG to the oracle's count
    m, gm, op, orc = make("BP3", 7, 1, shuffle=5)
    op.set_launch_shape(fem.F64, 6, 0)
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=4)
    xr, itr, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=1e-10)
    x = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
    st = op.cg(torch.from_numpy(b).cuda(), x, precond=fem.PC_JACOBI, rtol=1e-10)
    assert st["status"] == "FEM_OK" and abs(st["iterations"] - itr) <= 2
    assert rel(x.cpu().numpy(), xr) <= 1e-8
    # choice 6 exists for Gauss diffusion at p = 1 only
    for name, p in (("BP3", 2), ("BP5", 1), ("BP1", 1)):
        _, _, op2, _ = make(name, 2, p)
        with pytest.raises(fem.FemError):
            op2.set_launch_shape(fem.F64, 6, 0)


# ---------------------------------------------------------------- element-matrix body
@pytest.mark.parametrize("p,q,ncomp", [(1, 3, 1), (1, 2, 3), (2, 4, 1), (2, 3, 3)])
def test_element_matrix_body_matches_oracle(p, q, ncomp):
    # Gauss diffusion at p = 1, 2, one thread per element with the assembled
    # K_e (launch choice 7): 9^3 / 6^3 elements = several blocks of 128
    # threads with a ragged tail, shuffled order, both precisions
    n = 9 if p == 1 else 6
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=13, shuffle_seed=5)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, fem.DIFFUSION, fem.GAUSS, q, ncomp=ncomp, prec=fem.F32)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, q, ncomp=ncomp)
    for prec, tol in ((fem.F64, TOL64), (fem.F32, 1e-5)):
        for bps in (1, 0):
            op.set_launch_shape(prec, 7, bps)
            for x in inputs(m, ncomp, seed=q + 10 * p):
                xt = torch.from_numpy(x).cuda()
                if prec == fem.F64:
                    y = op.apply(xt).cpu().numpy()
                else:
                    y = op.apply_f32(xt.float()).double().cpu().numpy()
                assert rel(y, orc.apply(x)) <= tol, (prec, bps)
    # a listed subset of elements, and the empty list
    op.set_launch_shape(fem.F64, 7, 0)
    x = inputs(m, ncomp)[0]
    sel = np.random.default_rng(3).choice(m["E"], size=m["E"] // 3, replace=False).astype(np.int32)
    y = op.apply_elements(torch.from_numpy(sel).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, orc.apply(x, elems=sel)) <= TOL64
    y0 = op.apply_elements(torch.zeros(0, dtype=torch.int32, device="cuda"),
                           torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(y0 == 0.0)


def test_element_matrix_body_in_cg_and_only_where_valid():
    # the fused p^T A p of the element-matrix body drives CG to the oracle's
    # iteration count and solution (the default body at p = 1, 2 in FP64)
    for p, n in ((1, 7), (2, 4)):
        m, gm, op, orc = make("BP3", n, p, shuffle=6)
        op.set_launch_shape(fem.F64, 7, 0)
        b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=5)
        xr, itr, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=1e-10)
        x = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
        st = op.cg(torch.from_numpy(b).cuda(), x, precond=fem.PC_JACOBI, rtol=1e-10)
        assert st["status"] == "FEM_OK" and abs(st["iterations"] - itr) <= 2, (p, st, itr)
        assert rel(x.cpu().numpy(), xr) <= 1e-8
    # choice 7 exists for diffusion with a non-collocated rule at p = 1, 2 only
    for name, p in (("BP3", 3), ("BP5", 1), ("BP5", 2), ("BP1", 1)):
        _, _, op2, _ = make(name, 2, p)
        with pytest.raises(fem.FemError):
            op2.set_launch_shape(fem.F64, 7, 0)


@pytest.mark.parametrize("use_graph", [True, False])
def test_cg_zero_guess_ignores_x_and_matches_explicit_zero(use_graph):
    m, gm, op, orc = make("BP3", 4, 2, seed=6)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=9)).cuda()
    x0 = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
    st0 = op.cg(b, x0, rtol=1e-10, use_graph=use_graph)
    # garbage in x, zero_guess: the same solve as from an explicit zero
    x1 = torch.full_like(x0, 7.5)
    st1 = op.cg(b, x1, rtol=1e-10, use_graph=use_graph, zero_guess=True)
    assert st1["status"] == "FEM_OK" and abs(st1["iterations"] - st0["iterations"]) <= 1
    assert rel(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-9
    # fixed iteration count from zero: the oracle's iterate after 5 steps
    xr, _, _ = oracle.pcg(orc, b.cpu().numpy(), m["dirichlet"], rtol=0.0, maxit=5)
    x1.fill_(-3.0)
    st = op.cg(b, x1, rtol=0.0, maxit=5, use_graph=use_graph, zero_guess=True)
    assert st["iterations"] == 5 and rel(x1.cpu().numpy(), xr) <= 1e-10
    # the same buffers without the flag again: x is the initial guess once more
    st2 = op.cg(b, x1, rtol=1e-10, use_graph=use_graph)
    assert st2["iterations"] < st0["iterations"]
    assert rel(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-8

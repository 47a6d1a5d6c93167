"""GPU parity of the p-multigrid preconditioner (include/fem.h, fem_pmg_*)
against the FP64 oracle of oracle/pmg.py.

Transfers and the power-iteration estimate are compared directly; the
V-cycle is compared with the oracle's lmax passed to the GPU (oracle -> GPU,
never the reverse).  Tolerances: FP64 transfers 1e-13, lmax 1e-9, FP64
V-cycle 1e-10 (the coarse PCG and the Chebyshev recurrence amplify rounding
differences mildly), FP32 V-cycle 1e-4; the solve's residual is judged by
the oracle's apply.
"""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
from oracle import pmg as opmg
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _hierarchy(n, orders, prec=fem.F64, seed=3, coarse_dq=2, **kw):
    # the finest level is BP3 (q = p + 2); coarse levels use q = p + coarse_dq
    meshes = [fem_inputs.box_mesh(n, p, perturb=0.1, seed=seed) for p in orders]
    gms = [fem.Mesh(m) for m in meshes]
    ops = [fem.Operator(g, fem.DIFFUSION, fem.GAUSS, g.p + (2 if l == 0 else coarse_dq), prec=prec)
           for l, g in enumerate(gms)]
    pm = fem.Pmg(ops, prec=prec, **kw)
    levels = [opmg.Level(m, q=m["p"] + (2 if l == 0 else coarse_dq)) for l, m in enumerate(meshes)]
    return meshes, gms, ops, pm, levels


@pytest.mark.parametrize("orders", [(4, 2, 1), (8, 4), (3, 1), (5, 3, 2)])
def test_transfers_match_oracle(orders):
    meshes, gms, ops, pm, levels = _hierarchy(4, orders)
    rng = np.random.default_rng(1)
    for l in range(len(orders) - 1):
        xc = rng.uniform(-1, 1, levels[l + 1].N)
        rf = rng.uniform(-1, 1, levels[l].N)
        xf = pm.prolong(l, torch.from_numpy(xc).cuda()).cpu().numpy()
        rc = pm.restrict(l, torch.from_numpy(rf).cuda()).cpu().numpy()
        assert rel(xf, opmg.prolong(levels[l], levels[l + 1], xc)) <= 1e-13
        assert rel(rc, opmg.restrict(levels[l], levels[l + 1], rf)) <= 1e-13


def test_power_iteration_matches_oracle():
    meshes, gms, ops, pm, levels = _hierarchy(4, (4, 2, 1), power_its=20)
    for l in range(2):
        ref = opmg.power_lmax(levels[l], 20)
        assert abs(pm.lmax(l) - ref) <= 1e-9 * ref, (l, pm.lmax(l), ref)
    assert pm.lmax(2) == 0.0


@pytest.mark.parametrize("orders,degree,coarse_its",
                         [((4, 2, 1), 3, 20), ((4, 2, 1), 1, 1), ((6, 3, 1), 4, 10), ((2, 1), 2, 5)])
def test_vcycle_fp64_matches_oracle(orders, degree, coarse_its):
    meshes, gms, ops, pm, levels = _hierarchy(5, orders, cheb_degree=degree, coarse_its=coarse_its)
    lmax = [opmg.power_lmax(L, 20) for L in levels[:-1]] + [0.0]
    for l in range(len(orders) - 1):
        pm.set_lmax(l, lmax[l])
    rng = np.random.default_rng(2)
    r = np.where(levels[0].inner, rng.uniform(-1, 1, levels[0].N), 0.0)
    z = pm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    ref = opmg.vcycle(levels, lmax, r, degree=degree, coarse_its=coarse_its)
    assert rel(z, ref) <= 1e-10
    assert np.all(z[~levels[0].inner] == 0.0)


@pytest.mark.parametrize("orders", [(4, 2, 1), (8, 4, 2, 1)])
def test_vcycle_with_coarse_levels_on_p_plus_1_points_matches_oracle(orders):
    # coarse levels rediscretized with Gauss q = p + 1 (exact for affine bricks)
    meshes, gms, ops, pm, levels = _hierarchy(4, orders, coarse_dq=1, coarse_its=10)
    lmax = [opmg.power_lmax(L, 20) for L in levels[:-1]]
    for l in range(len(orders) - 1):
        pm.set_lmax(l, lmax[l])
    r = np.where(levels[0].inner, np.random.default_rng(11).uniform(-1, 1, levels[0].N), 0.0)
    z = pm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    ref = opmg.vcycle(levels, lmax + [0.0], r, degree=4, coarse_its=10)
    assert rel(z, ref) <= 1e-10


def test_vcycle_fp32_matches_oracle():
    meshes, gms, ops, pm, levels = _hierarchy(5, (4, 2, 1), prec=fem.F32, cheb_degree=4,
                                              coarse_its=10)
    lmax = [opmg.power_lmax(L, 20) for L in levels[:-1]]
    for l in range(2):
        pm.set_lmax(l, lmax[l])
    rng = np.random.default_rng(3)
    r = np.where(levels[0].inner, rng.uniform(-1, 1, levels[0].N), 0.0)
    z = pm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    ref = opmg.vcycle(levels, lmax + [0.0], r, degree=4, coarse_its=10)
    assert rel(z, ref) <= 1e-4


def test_single_level_is_the_coarse_pcg():
    m = fem_inputs.box_mesh(6, 2, perturb=0.1, seed=4)
    op = fem.Operator.bake_off(fem.Mesh(m), "BP3")
    pm = fem.Pmg([op], coarse_its=7)
    L = opmg.Level(m)
    r = np.where(L.inner, np.random.default_rng(5).uniform(-1, 1, L.N), 0.0)
    z = pm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel(z, opmg.coarse_pcg(L, r, 7)) <= 1e-11


@pytest.mark.parametrize("q", [2, 3])
@pytest.mark.parametrize("its", [1, 2, 9, 30])
def test_coarse_pcg_on_a_trilinear_level_matches_oracle(q, its):
    # the usual coarsest level (p = 1, Gauss q = 2 or 3); 11^3 elements span
    # several blocks
    m = fem_inputs.box_mesh(11, 1, perturb=0.1, seed=7, shuffle_seed=3)
    L = opmg.Level(m, q=q)
    r = np.where(L.inner, np.random.default_rng(its).uniform(-1, 1, L.N), 0.0)
    ref = opmg.coarse_pcg(L, r, its)
    for prec, tol in ((fem.F64, 1e-11), (fem.F32, 1e-4)):
        op = fem.Operator(fem.Mesh(m), fem.DIFFUSION, fem.GAUSS, q, prec=prec)
        pm = fem.Pmg([op], coarse_its=its, prec=prec)
        z = pm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel(z, ref) <= tol, (prec, rel(z, ref))
        z2 = pm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()   # graph replay
        assert rel(z2, ref) <= tol


@pytest.mark.parametrize("prec", [fem.F64, fem.F32])
def test_pmg_fcg_solves_to_1e10_in_few_iterations(prec):
    meshes, gms, ops, pm, levels = _hierarchy(8, (4, 2, 1), prec=prec)
    m0 = meshes[0]
    b = torch.from_numpy(fem_inputs.rhs_uniform(m0["N"], m0["dirichlet"], seed=6)).cuda()
    x = torch.zeros_like(b)
    st = pm.solve(b, x, rtol=1e-10)
    assert st["status"] == "FEM_OK"
    bn = np.where(levels[0].inner, b.cpu().numpy(), 0.0)
    res = np.where(levels[0].inner, bn - levels[0].op.apply(x.cpu().numpy()), 0.0)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(bn)
    x2 = torch.zeros_like(b)
    st2 = ops[0].cg(b, x2, precond=fem.PC_JACOBI, rtol=1e-10)
    assert st["iterations"] * 5 <= st2["iterations"], (st["iterations"], st2["iterations"])
    # replay of the captured graph gives the same count
    x3 = torch.zeros_like(b)
    st3 = pm.solve(b, x3, rtol=1e-10)
    assert abs(st3["iterations"] - st["iterations"]) <= 1


def test_pmg_rejects_inconsistent_hierarchies():
    ma = fem_inputs.box_mesh(3, 2, seed=1)
    mb = fem_inputs.box_mesh(4, 1, seed=1)
    oa = fem.Operator.bake_off(fem.Mesh(ma), "BP3")
    ob = fem.Operator.bake_off(fem.Mesh(mb), "BP3")
    with pytest.raises(fem.FemError):
        fem.Pmg([oa, ob])            # different element counts
    mc = fem_inputs.box_mesh(3, 3, seed=1)
    oc = fem.Operator.bake_off(fem.Mesh(mc), "BP3")
    with pytest.raises(fem.FemError):
        fem.Pmg([oa, oc])            # order not decreasing
    with pytest.raises(fem.FemError):
        fem.Pmg([oc, oa], prec=fem.F32)   # FP32 V-cycle needs FEM_F32 operators


def test_pmg_zero_rhs_and_a_single_element():
    # n = 1: the p = 1 level has no interior node (its coarse PCG sees an
    # empty system), the p = 2 level one; b = 0 needs no iteration
    meshes, gms, ops, pm, levels = _hierarchy(1, (4, 2, 1), coarse_its=5)
    lmax = [opmg.power_lmax(L, 20) for L in levels[:-1]]
    for l in range(2):
        pm.set_lmax(l, lmax[l])
    r = np.where(levels[0].inner, np.random.default_rng(9).uniform(-1, 1, levels[0].N), 0.0)
    z = pm.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    ref = opmg.vcycle(levels, lmax + [0.0], r, degree=4, coarse_its=5)
    assert rel(z, ref) <= 1e-10
    b = torch.zeros(meshes[0]["N"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st = pm.solve(b, x, rtol=1e-10)
    assert st["status"] == "FEM_OK" and st["iterations"] == 0
    assert torch.count_nonzero(x).item() == 0


def test_fp32_vcycle_as_preconditioner_of_refined_fcg():
    meshes, gms, ops, pm, levels = _hierarchy(8, (4, 2, 1), prec=fem.F32, coarse_dq=1)
    lmax = [opmg.power_lmax(L, 20) for L in levels[:-1]]
    for l in range(2):
        pm.set_lmax(l, lmax[l])
    # B(r) of the preconditioner object is the V-cycle, against the oracle
    rng = np.random.default_rng(8)
    r = np.where(levels[0].inner, rng.uniform(-1, 1, levels[0].N), 0.0)
    z = pm.vcycle_f32(torch.from_numpy(r).float().cuda()).double().cpu().numpy()
    assert rel(z, opmg.vcycle(levels, lmax + [0.0], r, degree=4, coarse_its=30)) <= 1e-4
    # refined FCG: FP64 true residual <= 1e-10 (oracle's apply), a couple of
    # refinement steps, about the iterations of the FP64 flexible CG
    m0 = meshes[0]
    b = torch.from_numpy(fem_inputs.rhs_uniform(m0["N"], m0["dirichlet"], seed=9)).cuda()
    x = torch.zeros_like(b)
    st = pm.solve_refined(b, x, rtol=1e-10, inner_rtol=1e-4)
    assert st["status"] == "FEM_OK" and st["true_rel"] <= 1e-10, st
    bn = np.where(levels[0].inner, b.cpu().numpy(), 0.0)
    res = np.where(levels[0].inner, bn - levels[0].op.apply(x.cpu().numpy()), 0.0)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(bn)
    assert 2 <= st["outer"] <= 4, st
    x2 = torch.zeros_like(b)
    st2 = pm.solve(b, x2, rtol=1e-10)
    assert st["iterations"] <= st2["iterations"] + 4, (st, st2)
    # a second solve replays the captured graph
    x3 = torch.zeros_like(b)
    st3 = pm.solve_refined(b, x3, rtol=1e-10, inner_rtol=1e-4)
    assert st3["true_rel"] <= 1e-10 and abs(st3["iterations"] - st["iterations"]) <= 1


def test_pmg_preconditioner_needs_fp32_hierarchy():
    meshes, gms, ops, pm, levels = _hierarchy(3, (2, 1), prec=fem.F64)
    with pytest.raises(fem.FemError):
        pm.solve_refined(torch.zeros(levels[0].N, dtype=torch.float64, device="cuda"),
                         torch.zeros(levels[0].N, dtype=torch.float64, device="cuda"))

"""GPU parity of the mixed-precision path against the FP64 oracle.

FP32 apply (FP32 qdata, FP32 arithmetic): relative l2 error <= 1e-5.
Refined solve (FP64 refinement around the FP32 inner PCG): the true FP64
residual of the returned x, measured by the oracle, is <= 1e-10 ||b||.
"""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def make(name, n, p, seed=7, shuffle=None):
    kind, ncomp, quad, dq = fem.BAKE_OFF[name]
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=seed, shuffle_seed=shuffle)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, kind, quad, p + dq, ncomp=ncomp, prec=fem.F32)
    orc = oracle.Operator(m, kind, quad, p + dq, ncomp=ncomp)
    return m, gm, op, orc


CASES = ([("BP3", p) for p in range(1, 9)] + [("BP5", p) for p in (1, 3, 7, 8)] +
         [("BP1", 2), ("BP1", 6), ("BP6", 7), ("BP2", 2), ("BP4", 1)])


@pytest.mark.parametrize("name,p", CASES)
def test_apply_f32_matches_oracle(name, p):
    n = {1: 5, 2: 4, 3: 3, 4: 3, 5: 2, 6: 2, 7: 2, 8: 2}[p]
    m, gm, op, orc = make(name, n, p, shuffle=5)
    x = np.random.default_rng(3).uniform(-1, 1, op.ncomp * m["N"])
    y = op.apply_f32(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    assert rel(y, orc.apply(x)) <= TOL32
    # the FP64 apply of an FP32 operator is still the FP64 one
    y64 = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y64, orc.apply(x)) <= 1e-12


@pytest.mark.parametrize("name,p,n", [("BP3", 2, 5), ("BP3", 5, 2), ("BP5", 7, 2), ("BP6", 3, 3)])
def test_refined_solve_reaches_fp64_residual(name, p, n):
    m, gm, op, orc = make(name, n, p)
    nc = op.ncomp
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=4, ncomp=nc)
    x = torch.zeros(nc * m["N"], dtype=torch.float64, device="cuda")
    st = op.solve_refined(torch.from_numpy(b).cuda(), x, rtol=1e-10, inner_rtol=1e-4)
    assert st["status"] == "FEM_OK", st
    assert st["outer"] >= 2 and st["true_rel"] <= 1e-10
    xs = x.cpu().numpy()
    inner = np.tile(m["dirichlet"] == 0, nc)
    res = np.where(inner, b - orc.apply(xs), 0.0)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(b) * 1.05
    xr, _, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=1e-12)
    assert rel(xs, xr) <= 1e-8
    # a second call (same buffers: the graph is replayed) gives the same answer
    # up to the order of the atomic additions
    bt = torch.from_numpy(b).cuda()
    x.zero_()
    st2 = op.solve_refined(bt, x, rtol=1e-10, inner_rtol=1e-4)
    st3 = op.solve_refined(bt, x.zero_(), rtol=1e-10, inner_rtol=1e-4)
    # FP32 atomics make the order of additions vary: counts agree to a few
    assert st3["true_rel"] <= 1e-10
    assert abs(st3["iterations"] - st2["iterations"]) <= max(6, 0.1 * st2["iterations"])
    assert rel(x.cpu().numpy(), xs) <= 1e-9


def test_refined_requires_f32_operator_and_limits_outer_steps():
    m = fem_inputs.box_mesh(3, 2, perturb=0.1, seed=1)
    gm = fem.Mesh(m)
    op64 = fem.Operator.bake_off(gm, "BP3")
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=1)).cuda()
    with pytest.raises(fem.FemError):
        op64.solve_refined(b, torch.zeros_like(b))
    op = fem.Operator.bake_off(gm, "BP3", prec=fem.F32)
    st = op.solve_refined(b, torch.zeros_like(b), rtol=1e-14, inner_rtol=0.5, max_outer=2)
    assert st["status"] == "FEM_ENOCONV" and st["outer"] <= 3


@pytest.mark.parametrize("name,p,n", [("BP3", 2, 14), ("BP3", 4, 11), ("BP5", 7, 9), ("BP3", 8, 6)])
def test_pipelined_fp32_apply_over_many_groups_per_block(name, p, n):
    # one block per SM: every block walks several element groups, so the
    # FP32 kernel's next-group column loads are exercised, and E is not a
    # multiple of the group size (ragged last group)
    m, gm, op, orc = make(name, n, p, shuffle=11)
    op.set_launch_shape(fem.F32, 0, 1)
    x = np.random.default_rng(8).uniform(-1, 1, op.ncomp * m["N"])
    y = op.apply_f32(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    assert rel(y, orc.apply(x)) <= TOL32

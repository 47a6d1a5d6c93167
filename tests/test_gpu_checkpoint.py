"""Checkpoint and resume of a CG solve (fem_cg_checkpoint / fem_cg_restore /
fem_cg_resume): a solve interrupted at iteration k, saved to host memory and
resumed -- on the same operator or on a fresh operator of the same mesh, as
in another process -- must reproduce the uninterrupted solve: the same
iteration count and the same solution up to the order of the apply's atomic
additions."""
import numpy as np
import pytest
import torch

import fem_inputs
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


@pytest.mark.parametrize("name,p,n,k,use_graph,fresh", [
    ("BP3", 3, 4, 17, True, False),
    ("BP3", 5, 3, 40, False, True),
    ("BP6", 2, 3, 25, True, True),
])
def test_interrupted_solve_resumes_as_if_uninterrupted(name, p, n, k, use_graph, fresh):
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=51, shuffle_seed=2)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, name)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=52,
                                                ncomp=op.ncomp)).cuda()
    x_ref = torch.zeros_like(b)
    st_ref = op.cg(b, x_ref, rtol=1e-10, use_graph=use_graph)
    assert st_ref["status"] == "FEM_OK" and st_ref["iterations"] > k
    x = torch.zeros_like(b)
    st1 = op.cg(b, x, rtol=1e-10, maxit=k, use_graph=use_graph)
    assert st1["status"] == "FEM_ENOCONV" and st1["iterations"] == k
    state = op.cg_checkpoint()
    x_saved = x.cpu().clone()
    if fresh:
        target = fem.Operator.bake_off(fem.Mesh(m), name)
        x = x_saved.cuda()
    else:
        target = op
        op.cg(b, torch.zeros_like(b), rtol=1e-10, maxit=3)   # the workspace is reused ...
    target.cg_restore(state)                                  # ... and restored
    st2 = target.cg_resume(b, x, rtol=1e-10)
    assert st2["status"] == "FEM_OK"
    assert st2["iterations"] == st_ref["iterations"]
    assert rel(x, x_ref) <= 1e-12
    assert abs(st2["rnorm"] - st_ref["rnorm"]) <= 1e-2 * st_ref["rnorm"]


def test_fixed_count_solve_resumes_and_bad_states_are_refused():
    m = fem_inputs.box_mesh(4, 2, perturb=0.1, seed=53)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, "BP1")
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=54)).cuda()
    x_ref = torch.zeros_like(b)
    op.cg(b, x_ref, precond=fem.PC_NONE, maxit=100, rtol=0.0)
    x = torch.zeros_like(b)
    op.cg(b, x, precond=fem.PC_NONE, maxit=60, rtol=0.0)
    st = op.cg_resume(b, x, precond=fem.PC_NONE, maxit=40, rtol=0.0)
    assert st["iterations"] == 100 and rel(x, x_ref) <= 1e-12
    with pytest.raises(fem.FemError):
        op.cg_resume(b, x, precond=fem.PC_JACOBI, maxit=5, rtol=0.0)   # other preconditioner
    op.cg(b, x, precond=fem.PC_JACOBI, rtol=1e-10)                      # converged, not capped
    with pytest.raises(fem.FemError):
        op.cg_resume(b, x, precond=fem.PC_JACOBI)
    state = op.cg_checkpoint()
    other = fem.Operator.bake_off(fem.Mesh(fem_inputs.box_mesh(3, 2, perturb=0.1, seed=1)), "BP1")
    with pytest.raises(fem.FemError):
        other.cg_restore(state)                                         # wrong size
    bad = state.copy()
    bad[:8] = 0
    with pytest.raises(fem.FemError):
        op.cg_restore(bad)

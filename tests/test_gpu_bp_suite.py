"""The vector bake-off problems as solves (BP2: vector mass, BP4: vector
diffusion with Gauss q = p+2; section "Benchmarks"): FP64 CG on the GPU
against the oracle's numpy CG on the same system.  Iteration counts within
2, solutions within 1e-8 relative (CG iterates differ by rounding order)."""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("name,p,n", [("BP2", 3, 4), ("BP4", 3, 4), ("BP4", 5, 3), ("BP6", 4, 3)])
def test_vector_bp_solve_matches_oracle_cg(name, p, n):
    kind, nc, quad, dq = fem.BAKE_OFF[name]
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=11)
    op = fem.Operator.bake_off(fem.Mesh(m), name)
    okind = oracle.MASS if kind == fem.MASS else oracle.DIFFUSION
    oquad = oracle.GAUSS if quad == fem.GAUSS else oracle.LOBATTO
    orc = oracle.Operator(m, okind, oquad, p + dq, ncomp=nc)
    b = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=12, ncomp=nc)
    pc = "none" if kind == fem.MASS else "jacobi"
    xr, kr, _ = oracle.pcg(orc, b, m["dirichlet"], rtol=1e-10, precond=pc)
    x = torch.zeros(nc * m["N"], dtype=torch.float64, device="cuda")
    st = op.cg(torch.from_numpy(b).cuda(), x, precond=fem.PC_NONE if pc == "none" else fem.PC_JACOBI,
               rtol=1e-10)
    assert st["status"] == "FEM_OK"
    assert abs(st["iterations"] - kr) <= 2, (st["iterations"], kr)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xr) <= 1e-8 * np.linalg.norm(xr)

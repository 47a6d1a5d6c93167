"""The double-word bodies of the FP64 apply (launch choices 8..11).

These bodies carry every contraction and pointwise product of the FP64
operator in double-word arithmetic (pairs of FP32 numbers) on the FP32 pipe.
They must meet the FP64 bar: the oracle's result to 1e-12 relative l2 on
every bake-off problem and order, for random and smooth input vectors, on
shuffled meshes with a ragged last element group, for element subsets, and
inside CG (iterations and solution as the oracle's PCG).
"""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu

DW_LINES = (8, 9, 10, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23)   # 12..14 pipelined gather, 15..17 packed f32x2, 18..23 packed with L2 prefetch (21..23 and the pipelined gather)
DW_ELMAT = 11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def dw_choices(kind, quad, p, colloc):
    out = [] if (kind == fem.MASS and colloc) else list(DW_LINES)
    if kind == fem.DIFFUSION and quad == fem.GAUSS and p <= 2:
        out.append(DW_ELMAT)
    return out


CASES = [("BP1", p, n) for p, n in ((1, 7), (2, 5), (3, 3), (5, 2), (8, 2))] + \
        [("BP2", 2, 3), ("BP4", 3, 2), ("BP6", 4, 2)] + \
        [("BP3", p, n) for p, n in ((1, 7), (2, 5), (3, 4), (4, 3), (5, 3), (6, 2), (7, 2), (8, 2))] + \
        [("BP5", p, n) for p, n in ((1, 6), (2, 4), (3, 3), (4, 3), (5, 2), (6, 2), (7, 2), (8, 2))]


@pytest.mark.parametrize("name,p,n", CASES)
def test_dw_apply_matches_oracle(name, p, n):
    kind, ncomp, quad, dq = fem.BAKE_OFF[name]
    q = p + dq
    colloc = quad == fem.LOBATTO and q == p + 1
    # n^3 elements, shuffled: the last element group of every block size is ragged
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=31 + p, shuffle_seed=7)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, kind, quad, q, ncomp=ncomp)
    orc = oracle.Operator(m, kind, quad, q, ncomp=ncomp)
    rng = np.random.default_rng(5)
    xr = rng.uniform(-1, 1, ncomp * m["N"])
    # a smooth field on the node lattice
    M = m["M"]
    g = np.arange(m["N"])
    I, J, K = g % M, (g // M) % M, g // (M * M)
    t = np.pi / max(M - 1, 1)
    xs = np.tile(np.sin(t * I) * np.sin(2 * t * J) * np.cos(t * K), ncomp)
    refs = [(xr, orc.apply(xr)), (xs, orc.apply(xs))]
    for choice in dw_choices(kind, quad, p, colloc):
        for bps in (1, 0):
            op.set_launch_shape(fem.F64, choice, bps)
            for x, ref in refs:
                y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
                assert rel(y, ref) <= 1e-12, (choice, bps, rel(y, ref))


def test_dw_rejected_where_it_does_not_exist():
    m = fem_inputs.box_mesh(2, 3, perturb=0.1, seed=3)
    gm = fem.Mesh(m)
    op3 = fem.Operator.bake_off(gm, "BP3", prec=fem.F32)
    with pytest.raises(fem.FemError):
        op3.set_launch_shape(fem.F32, 8, 0)          # FP32 has no double-word body
    with pytest.raises(fem.FemError):
        op3.set_launch_shape(fem.F64, DW_ELMAT, 0)   # no element matrices at p = 3
    mc = fem.Operator(gm, fem.MASS, fem.LOBATTO, 4)  # collocated mass: pointwise only
    with pytest.raises(fem.FemError):
        mc.set_launch_shape(fem.F64, 8, 0)


@pytest.mark.parametrize("p,choice", [(2, DW_ELMAT), (4, 8), (7, 9)])
def test_dw_element_subsets(p, choice):
    m = fem_inputs.box_mesh(3, p, perturb=0.1, seed=8, shuffle_seed=3)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, "BP3")
    op.set_launch_shape(fem.F64, choice, 0)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, p + 2)
    x = np.random.default_rng(2).uniform(-1, 1, m["N"])
    elems = np.random.default_rng(4).choice(m["E"], size=m["E"] // 2 + 1, replace=False).astype(np.int32)
    ref = orc.apply(x, elems=elems)
    y = op.apply_elements(torch.from_numpy(elems).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) <= 1e-12
    y0 = op.apply_elements(torch.zeros(0, dtype=torch.int32, device="cuda"),
                           torch.from_numpy(x).cuda()).cpu().numpy()
    assert not y0.any()


@pytest.mark.parametrize("name,p,n,choice", [("BP3", 1, 6, DW_ELMAT), ("BP3", 2, 4, DW_ELMAT),
                                             ("BP3", 4, 3, 8), ("BP5", 6, 2, 8),
                                             ("BP6", 3, 2, 8)])
def test_dw_pcg_matches_oracle(name, p, n, choice):
    kind, ncomp, quad, dq = fem.BAKE_OFF[name]
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=12, shuffle_seed=1)
    gm = fem.Mesh(m)
    op = fem.Operator(gm, kind, quad, p + dq, ncomp=ncomp)
    op.set_launch_shape(fem.F64, choice, 0)
    orc = oracle.Operator(m, kind, quad, p + dq, ncomp=ncomp)
    bn = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=13, ncomp=ncomp)
    xo, it_o, _ = oracle.pcg(orc, bn, m["dirichlet"], rtol=1e-10)
    x = torch.zeros(ncomp * m["N"], dtype=torch.float64, device="cuda")
    st = op.cg(torch.from_numpy(bn).cuda(), x, rtol=1e-10)
    assert st["status"] == "FEM_OK"
    assert abs(st["iterations"] - it_o) <= 2
    assert rel(x.cpu().numpy(), xo) <= 1e-8

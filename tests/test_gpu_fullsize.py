"""GPU parity at the benchmark's full sizes, in the launch configuration
bench.py times: the whole-mesh apply is computed on the GPU and sampled rows
are checked against the FP64 oracle, which computes each sampled row from the
elements that contain that node (index arithmetic on the brick lattice).

Sizes: BP3 (Gauss q = p+2) for p = 1..8 at about 5e7 DOFs each; BP5 / BP6
(Gauss-Lobatto, p = 7, n = 44, 29.5M nodes per component).  Tolerances: FP64
1e-12, FP32 1e-5 relative l2 over the sampled rows.
"""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu

NROWS = 1024


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def _rows(m, seed):
    rng = np.random.default_rng(seed)
    rows = rng.choice(m["N"], NROWS, replace=False)
    # include the first and last nodes (corners) and an interior lattice line
    return np.unique(np.concatenate([rows, [0, m["N"] - 1, m["N"] // 2]]))


def _check(m, gm, name, p, rows, seed):
    kind, ncomp, quad, dq = fem.BAKE_OFF[name]
    op = fem.Operator(gm, kind, quad, p + dq, ncomp=ncomp, prec=fem.F32)
    orc = oracle.Operator(m, kind, quad, p + dq)
    x = np.random.default_rng(seed).uniform(-1, 1, ncomp * m["N"])
    xt = torch.from_numpy(x).cuda()
    y64 = op.apply(xt)
    y32 = op.apply_f32(xt.float())
    ptr, el = fem_inputs.elements_of_nodes(m, rows)
    N = m["N"]
    for c in range(ncomp):
        ref = orc.apply_rows(x[c * N:(c + 1) * N], rows, ptr, el)
        g64 = y64[c * N:(c + 1) * N].cpu().numpy()[rows]
        g32 = y32[c * N:(c + 1) * N].double().cpu().numpy()[rows]
        e64 = np.linalg.norm(g64 - ref) / np.linalg.norm(ref)
        e32 = np.linalg.norm(g32 - ref) / np.linalg.norm(ref)
        assert e64 <= 1e-12, (name, p, c, e64)
        assert e32 <= 1e-5, (name, p, c, e32)


@pytest.mark.parametrize("p", range(1, 9))
def test_bp3_full_size_sampled_rows(p):
    n = fem_inputs.bp3_mesh_n(5e7, p)
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=100 + p)
    gm = fem.Mesh(m)
    _check(m, gm, "BP3", p, _rows(m, p), seed=200 + p)


def test_bp5_bp6_full_size_sampled_rows():
    m = fem_inputs.box_mesh(44, 7, perturb=0.1, seed=500)
    gm = fem.Mesh(m)
    rows = _rows(m, 7)
    _check(m, gm, "BP5", 7, rows, seed=1)
    _check(m, gm, "BP6", 7, rows, seed=2)

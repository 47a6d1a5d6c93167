"""GPU operators on meshes whose elements have arbitrary (right-handed)
local frames, numbered by fem_mesh_connectivity: the fused apply against the
FP64 oracle on the same mesh (1e-12), and a BP3 solve against the solve on
the lexicographic mesh at the same physical nodes (1e-8)."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,p", [("BP3", 4), ("BP3", 7), ("BP1", 3), ("BP5", 5)])
def test_apply_on_rotated_frames_matches_oracle(name, p):
    m = fem_inputs.box_mesh(4, p, perturb=0.1, seed=21, shuffle_seed=3)
    r = fem_inputs.rotate_elements(m, seed=22)
    c = fem.mesh_connectivity(p, r["vert_xyz"], r["elem_verts"])
    kind, nc, quad, dq = fem.BAKE_OFF[name]
    op = fem.Operator.bake_off(fem.Mesh(c), name, prec=fem.F32)
    orc = oracle.Operator(c, oracle.MASS if kind == fem.MASS else oracle.DIFFUSION,
                          oracle.GAUSS if quad == fem.GAUSS else oracle.LOBATTO, p + dq)
    x = np.random.default_rng(4).uniform(-1, 1, c["N"])
    y64 = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    y32 = op.apply_f32(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    ref = orc.apply(x)
    assert rel(y64, ref) <= 1e-12
    assert rel(y32, ref) <= 1e-5


def test_solution_does_not_depend_on_element_frames():
    p = 3
    m = fem_inputs.box_mesh(5, p, perturb=0.1, seed=23)
    r = fem_inputs.rotate_elements(m, seed=24)
    c = fem.mesh_connectivity(p, r["vert_xyz"], r["elem_verts"])
    xm = oracle.nodes_from_vertices(m)
    xc = oracle.nodes_from_vertices(c)
    key = lambda X: [tuple(k) for k in np.round(X * 1e9).astype(np.int64)]
    pos = {k: i for i, k in enumerate(key(xm))}
    perm = np.array([pos[k] for k in key(xc)])
    f = np.where(m["dirichlet"] == 0, np.cos(3 * xm[:, 0]) * xm[:, 1] + xm[:, 2], 0.0)
    sols = []
    for mesh, b in ((m, f), (c, f[perm])):
        op = fem.Operator.bake_off(fem.Mesh(mesh), "BP3")
        x = torch.zeros(mesh["N"], dtype=torch.float64, device="cuda")
        st = op.cg(torch.from_numpy(b).cuda(), x, precond=fem.PC_JACOBI, rtol=1e-12)
        assert st["status"] == "FEM_OK"
        sols.append(x.cpu().numpy())
    assert rel(sols[1], sols[0][perm]) <= 1e-8

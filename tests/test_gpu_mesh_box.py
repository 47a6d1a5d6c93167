"""The library's bake-off mesh generator (fem_mesh_box) on the GPU.

The Cartesian mesh (perturb = 0) must be the one fem_inputs.box_mesh builds
(same numbering, same node coordinates); the perturbed mesh is rebuilt here
on the host from the published SplitMix64 definition (the generator the
library documents) and the library's BP3 operator on it must match the FP64
oracle on that rebuilt mesh.  Plus the geometric facts: boundary nodes on
the cube's faces, vertex moves bounded by perturb * h, the mass operator
integrating 1 to the volume 1 and diffusion annihilating constants.
"""
import numpy as np
import pytest
import torch

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu

MASK = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fembuild.build()
    assert torch.cuda.is_available()


def splitmix64_at(seed, i):
    """SplitMix64 output i of a generator whose state starts at `seed`
    (Steele, Lea & Flood 2014), in Python integers."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def host_box(p, n, perturb, seed):
    """fem_inputs' Cartesian mesh with the vertices moved as fem_mesh_box
    documents."""
    m = fem_inputs.box_mesh(n, p, perturb=0.0)
    v = m["vert_xyz"].copy()
    nv = n + 1
    h = 1.0 / n
    for vid in range(v.shape[0]):
        idx = (vid % nv, (vid // nv) % nv, vid // (nv * nv))
        for d in range(3):
            if 0 < idx[d] < n:
                u = (splitmix64_at(seed, 3 * vid + d) >> 11) * 2.0 ** -53
                v[vid, d] += perturb * h * (2.0 * u - 1.0)
    m["vert_xyz"] = v
    return m


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("p,n", [(1, 4), (3, 3), (5, 2)])
def test_cartesian_box_is_fem_inputs_mesh(p, n):
    gm = fem.Mesh.box(p, n, perturb=0.0)
    m = fem_inputs.box_mesh(n, p, perturb=0.0)
    assert (gm.N, gm.E) == (m["N"], m["E"])
    xyz = oracle.nodes_from_vertices(m)
    assert np.max(np.abs(gm.node_xyz - xyz)) <= 1e-15
    op = fem.Operator.bake_off(gm, "BP3")
    x = np.random.default_rng(3).uniform(-1, 1, m["N"])
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, p + 2).apply(x)
    assert rel(y, ref) <= 1e-12


@pytest.mark.parametrize("p,n,seed", [(2, 4, 0), (4, 3, 12345), (7, 2, 2 ** 63 + 5)])
def test_perturbed_box_matches_oracle_on_the_documented_mesh(p, n, seed):
    gm = fem.Mesh.box(p, n, perturb=0.1, seed=seed)
    m = host_box(p, n, 0.1, seed)
    xyz = gm.node_xyz
    assert np.max(np.abs(xyz - oracle.nodes_from_vertices(m))) <= 1e-15
    for name, kind, quad in (("BP3", oracle.DIFFUSION, oracle.GAUSS),
                             ("BP1", oracle.MASS, oracle.GAUSS),
                             ("BP5", oracle.DIFFUSION, oracle.LOBATTO)):
        op = fem.Operator.bake_off(gm, name)
        q = p + (1 if quad == oracle.LOBATTO else 2)
        x = np.random.default_rng(4).uniform(-1, 1, m["N"])
        y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert rel(y, oracle.Operator(m, kind, quad, q).apply(x)) <= 1e-12, name


def test_box_geometry_facts():
    p, n = 3, 4
    a = fem.Mesh.box(p, n, perturb=0.2, seed=7)
    b = fem.Mesh.box(p, n, perturb=0.2, seed=7)
    c = fem.Mesh.box(p, n, perturb=0.2, seed=8)
    assert np.array_equal(a.node_xyz, b.node_xyz)
    assert not np.array_equal(a.node_xyz, c.node_xyz)
    xyz = a.node_xyz
    M = p * n + 1
    g = np.arange(a.N)
    I, J, K = g % M, (g // M) % M, g // (M * M)
    for d, idx in enumerate((I, J, K)):
        assert np.all(xyz[idx == 0, d] == 0.0) and np.all(xyz[idx == M - 1, d] == 1.0)
    # vertices (every p-th node line) move by at most perturb * h
    cart = oracle.nodes_from_vertices(fem_inputs.box_mesh(n, p, perturb=0.0))
    vtx = (I % p == 0) & (J % p == 0) & (K % p == 0)
    assert np.max(np.abs(xyz[vtx] - cart[vtx])) <= 0.2 / n + 1e-15
    assert np.max(np.abs(xyz[vtx] - cart[vtx])) > 0.05 / n
    one = torch.ones(a.N, dtype=torch.float64, device="cuda")
    mass = fem.Operator.bake_off(a, "BP1")
    assert abs(torch.dot(one, mass.apply(one)).item() - 1.0) <= 1e-12
    diff = fem.Operator.bake_off(a, "BP3")
    scale = torch.linalg.norm(diff.apply(torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, a.N)).cuda())).item()
    assert torch.linalg.norm(diff.apply(one)).item() <= 1e-12 * scale

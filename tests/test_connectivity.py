"""Q_p connectivity from a hexahedral vertex list (fem_mesh_connectivity,
host code of the library) against geometry: two (element, local node) pairs
must get the same global id exactly when the trilinear map puts them at the
same point, Dirichlet nodes are the nodes on the cube's surface, and the
operator does not depend on the elements' local frames.  CPU only."""
import ctypes

import numpy as np
import pytest

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem


def local_node_coords(m):
    """[E, P^3, 3]: x(xi_a) = sum_v N_v(xi_a) X_v with trilinear N_v and the
    Gauss-Lobatto nodes xi of order p (computed here, not by the library)."""
    p = m["p"]; P = p + 1
    z, _ = oracle.gauss_lobatto(P)
    c, b, a = np.meshgrid(np.arange(P), np.arange(P), np.arange(P), indexing="ij")
    xi = np.stack([z[a.ravel()], z[b.ravel()], z[c.ravel()]], axis=1)       # [P^3, 3]
    Nv = np.ones((P ** 3, 8))
    for v in range(8):
        for d, bit in enumerate(((v >> 0) & 1, (v >> 1) & 1, (v >> 2) & 1)):
            Nv[:, v] *= 0.5 * (1 + xi[:, d]) if bit else 0.5 * (1 - xi[:, d])
    X = m["vert_xyz"][m["elem_verts"]]                                      # [E, 8, 3]
    return np.einsum("av,evd->ead", Nv, X)


def check_against_geometry(c):
    xyz = local_node_coords(c).reshape(-1, 3)
    ids = c["elem_nodes"].ravel()
    N = c["N"]
    assert ids.min() == 0 and ids.max() == N - 1 and np.unique(ids).size == N
    # same id -> same point
    ref = np.zeros((N, 3))
    ref[ids] = xyz
    assert np.abs(ref[ids] - xyz).max() <= 1e-13
    # different ids -> different points
    keys = np.round(ref * 1e9).astype(np.int64)
    assert np.unique(keys, axis=0).shape[0] == N
    on_surface = np.any((np.abs(ref) < 1e-12) | (np.abs(ref - 1.0) < 1e-12), axis=1)
    np.testing.assert_array_equal(c["dirichlet"].astype(bool), on_surface)
    return ref


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("rotate", [False, True])
def test_connectivity_matches_geometry(p, rotate):
    n = 3 if p <= 4 else 2
    m = fem_inputs.box_mesh(n, p, perturb=0.15, seed=p, shuffle_seed=p + 10)
    src = fem_inputs.rotate_elements(m, seed=p) if rotate else m
    c = fem.mesh_connectivity(p, src["vert_xyz"], src["elem_verts"])
    assert c["N"] == m["N"]
    check_against_geometry(c)


def test_rotations_are_the_24_proper_cube_symmetries():
    R = fem_inputs.cube_rotations()
    assert len(R) == 24
    assert len({r.tobytes() for r in R}) == 24
    for r in R:
        assert np.array_equal(r @ r.T, np.eye(3, dtype=np.int64)) and round(np.linalg.det(r)) == 1


@pytest.mark.parametrize("p", [2, 3])
def test_operator_does_not_depend_on_element_frames(p):
    # the oracle's operator on the rotated mesh (library connectivity) and on
    # the original mesh agree at the same physical nodes
    m = fem_inputs.box_mesh(3, p, perturb=0.1, seed=7)
    r = fem_inputs.rotate_elements(m, seed=8)
    c = fem.mesh_connectivity(p, r["vert_xyz"], r["elem_verts"])
    xr = check_against_geometry(c)
    xm = oracle.nodes_from_vertices(m)
    # map rotated-mesh node ids to original ids by position
    key = lambda X: [tuple(k) for k in np.round(X * 1e9).astype(np.int64)]
    pos = {k: i for i, k in enumerate(key(xm))}
    perm = np.array([pos[k] for k in key(xr)])
    f = lambda X: np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] ** 2
    A0 = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, p + 2)
    A1 = oracle.Operator(c, oracle.DIFFUSION, oracle.GAUSS, p + 2)
    y0 = A0.apply(f(xm))
    y1 = A1.apply(f(xr))
    np.testing.assert_allclose(y1, y0[perm], atol=1e-12 * np.abs(y0).max())


def test_connectivity_rejects_bad_meshes():
    m = fem_inputs.box_mesh(2, 2, seed=1)
    ev = m["elem_verts"].copy()
    ev[0, 3] = ev[0, 2]
    with pytest.raises(fem.FemError, match="repeats vertex"):
        fem.mesh_connectivity(2, m["vert_xyz"], ev)
    ev = m["elem_verts"].copy()
    ev[1, 0] = m["vert_xyz"].shape[0]
    with pytest.raises(fem.FemError, match="out of range"):
        fem.mesh_connectivity(2, m["vert_xyz"], ev)
    ev = np.concatenate([m["elem_verts"], m["elem_verts"][:1]])   # element 0 twice: faces of 3
    with pytest.raises(fem.FemError, match="more than two"):
        fem.mesh_connectivity(2, m["vert_xyz"], ev)
    with pytest.raises(fem.FemError):
        fem.mesh_connectivity(0, m["vert_xyz"], m["elem_verts"])

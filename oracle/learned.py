"""FP64 oracle of the learned preconditioner's apply (TEST INFRASTRUCTURE).

The paper has no learned preconditioner; its preconditioning material is
the section "Ecosystem" (matrix-free preconditioning).  The map built here is
the one the library defines (a Jacobi term plus a per-element network
correction, averaged over the elements that share a node):

    z = D^{-1} r + gamma * sum_e G_e^T ( w * ||r_e|| * net([r_e / ||r_e||, g_e])[:P^3] )

where r_e = G_e r are the element's P^3 values of r, ||.|| the Euclidean
norm over them (a zero norm gives a zero network input for r_e and a zero
correction), g_e the element's 32 geometric features, w = 1 / (number of
elements that hold the node), D^{-1} the inverse diagonal of the operator on
interior nodes (0 on Dirichlet nodes), and the correction is not added on
Dirichlet nodes.  Features g_e: the offsets of the element's 8 corner nodes
from their centroid divided by h = (2/sqrt 3) * (root-mean-square corner
distance) -- the side of a cube with those corners -- then log kappa at the
8 corners (0 without a coefficient).

Everything is written out per element in FP64 numpy, around the FP64
network forward of oracle/mlp.c.  Only tests import this module.
"""
import numpy as np

from . import mlp_forward, nodes_from_vertices

NUM_FEAT = 32


def multiplicity_weights(mesh):
    """w[i] = 1 / (number of elements holding node i), 0 for unused nodes."""
    cnt = np.bincount(np.asarray(mesh["elem_nodes"]).ravel(), minlength=mesh["N"]).astype(np.float64)
    return np.where(cnt > 0, 1.0 / np.where(cnt > 0, cnt, 1.0), 0.0)


def corner_locals(P):
    """Local node ids of the 8 corners, corner v = (v & 1, v & 2, v & 4)."""
    out = []
    for v in range(8):
        a = P - 1 if v & 1 else 0
        b = P - 1 if v & 2 else 0
        c = P - 1 if v & 4 else 0
        out.append(a + P * b + P * P * c)
    return out


def features(mesh, rff=None, sigma=1.0, node_xyz=None):
    """[E][32] element features g_e (see the module docstring)."""
    xyz = nodes_from_vertices(mesh) if node_xyz is None else node_xyz
    P = mesh["p"] + 1
    en = np.asarray(mesh["elem_nodes"])
    cl = corner_locals(P)
    E = mesh["E"]
    g = np.zeros((E, NUM_FEAT))
    for e in range(E):
        c = xyz[en[e, cl]]                       # [8][3]
        cen = c.mean(axis=0)
        off = c - cen
        rms = np.sqrt(np.sum(off * off) / 8.0)
        h = 2.0 / np.sqrt(3.0) * rms
        g[e, :24] = (off / h).ravel()
        if rff is not None:
            M = rff.shape[0]
            for v in range(8):
                arg = rff[:, :3] @ c[v] + rff[:, 3]
                g[e, 24 + v] = sigma * np.sqrt(2.0 / M) * np.sum(np.cos(arg))
    return g


def precond_apply(mesh, diag, dims, params, r, gamma, feat):
    """z = B(r) in FP64 (see the module docstring).

    diag: the operator's diagonal [N]; dims = (n_in, n_h, n_out); params:
    the network's flat parameter array; r: [N]; feat: [E][32]."""
    n_in, n_h, n_out = dims
    P = mesh["p"] + 1
    P3 = P ** 3
    en = np.asarray(mesh["elem_nodes"])
    inner = np.asarray(mesh["dirichlet"]) == 0
    dinv = np.where(inner, 1.0 / np.where(inner, diag, 1.0), 0.0)
    z = dinv * r
    if gamma == 0.0:
        return z
    w = multiplicity_weights(mesh)
    E = mesh["E"]
    X = np.zeros((E, n_in))
    norms = np.zeros(E)
    for e in range(E):
        re = r[en[e]]
        nr = np.sqrt(np.sum(re * re))
        norms[e] = nr
        X[e, :P3] = re / nr if nr > 0 else 0.0
        X[e, P3:P3 + NUM_FEAT] = feat[e]
    Y, _, _ = mlp_forward(dims, params, X)
    corr = np.zeros_like(z)
    for e in range(E):
        for a in range(P3):
            i = en[e, a]
            corr[i] += w[i] * norms[e] * Y[e, a]
    return z + gamma * np.where(inner, corr, 0.0)

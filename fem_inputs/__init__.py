"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds NO arithmetic of the finite element method: it lays out a
structured brick mesh of the unit cube (vertex grid, perturbation, element and
node numbering), draws random right-hand sides and the random parameters of
the coefficient field.  Both the oracle and the CUDA library consume these
arrays; neither side's arithmetic lives here.

Workload shapes follow the bake-off problems (section "Benchmarks"): the unit
cube split into n^3 hexahedra whose interior vertices are moved by up to 0.1 h
(seeded), Q_p elements, global nodes numbered lexicographically on the
(p n + 1)^3 node lattice, homogeneous Dirichlet nodes on the cube's surface.
"""
import numpy as np

__all__ = ["box_mesh", "rhs_uniform", "rff_params", "elements_of_nodes",
           "bp3_mesh_n", "batch_problems", "mlp_init"]


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def box_mesh(n, p, perturb=0.1, seed=0, shuffle_seed=None):
    """Structured n x n x n brick mesh of [0,1]^3 with Q_p connectivity.

    Returns a dict with
      vert_xyz   [(n+1)^3, 3] float64, vertex v = i + (n+1)(j + (n+1)k);
                 every interior vertex coordinate is moved by U(-perturb h,
                 perturb h), boundary vertices stay on the cube's faces;
      elem_verts [E, 8] int32, vertex (vi,vj,vk) of an element at vi + 2vj + 4vk;
      elem_nodes [E, (p+1)^3] int32, local node (a,b,c) at a + P b + P^2 c,
                 global node (I,J,K) = I + M (J + M K), M = p n + 1;
      dirichlet  [N] uint8, 1 on the cube's surface;
      perm       element permutation applied (identity unless shuffled);
      n, p, N, E, M.
    """
    n = int(n); p = int(p)
    if n < 1 or p < 1:
        raise ValueError("n and p must be >= 1")
    P = p + 1
    nv = n + 1
    M = p * n + 1
    N = M ** 3
    E = n ** 3
    h = 1.0 / n
    g = np.arange(nv, dtype=np.float64) * h
    k, j, i = np.meshgrid(np.arange(nv), np.arange(nv), np.arange(nv), indexing="ij")
    vert = np.stack([g[i.ravel()], g[j.ravel()], g[k.ravel()]], axis=1)
    if perturb > 0:
        rng = _rng(seed)
        delta = rng.uniform(-perturb * h, perturb * h, size=vert.shape)
        for d, idx in enumerate((i.ravel(), j.ravel(), k.ravel())):
            on_face = (idx == 0) | (idx == n)
            delta[on_face, d] = 0.0
        vert = vert + delta
    del i, j, k
    ez, ey, ex = np.meshgrid(np.arange(n, dtype=np.int64), np.arange(n, dtype=np.int64),
                             np.arange(n, dtype=np.int64), indexing="ij")
    ex = ex.ravel(); ey = ey.ravel(); ez = ez.ravel()
    ev = np.empty((E, 8), dtype=np.int32)
    for v in range(8):
        vi, vj, vk = v & 1, (v >> 1) & 1, (v >> 2) & 1
        ev[:, v] = (ex + vi) + nv * ((ey + vj) + nv * (ez + vk))
    loc = np.arange(P)
    cc, bb, aa = np.meshgrid(loc, loc, loc, indexing="ij")
    aa = aa.ravel(); bb = bb.ravel(); cc = cc.ravel()
    base = (p * ex) + M * ((p * ey) + M * (p * ez))
    offs = aa + M * (bb + M * cc)
    en = np.empty((E, P ** 3), dtype=np.int32)
    chunk = max(1, (1 << 24) // (P ** 3))
    for s in range(0, E, chunk):
        en[s:s + chunk] = (base[s:s + chunk, None] + offs[None, :]).astype(np.int32)
    del base, ex, ey, ez
    mk, mj, mi = np.meshgrid(np.arange(M), np.arange(M), np.arange(M), indexing="ij")
    bnd = ((mi == 0) | (mi == M - 1) | (mj == 0) | (mj == M - 1) | (mk == 0) | (mk == M - 1))
    dirichlet = bnd.ravel().astype(np.uint8)
    del mi, mj, mk, bnd
    perm = np.arange(E, dtype=np.int64)
    if shuffle_seed is not None:
        perm = _rng(shuffle_seed).permutation(E)
        ev = np.ascontiguousarray(ev[perm])
        en = np.ascontiguousarray(en[perm])
    return dict(vert_xyz=np.ascontiguousarray(vert), elem_verts=ev, elem_nodes=en,
                dirichlet=dirichlet, perm=perm, n=n, p=p, N=N, E=E, M=M)


def cube_rotations():
    """The 24 proper rotations of the cube as 3x3 signed permutation matrices
    (det +1)."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r, c in enumerate(perm):
                R[r, c] = signs[r]
            if round(np.linalg.det(R)) == 1:
                out.append(R)
    return out


def rotate_elements(mesh, seed):
    """The same mesh with each element's local frame turned by a seeded
    proper rotation of the cube: elem_verts [E, 8] are permuted so that new
    local vertex c' (c' in {0,1}^3, index i + 2j + 4k) is the old vertex at
    (R (2c' - 1) + 1) / 2.  elem_nodes and dirichlet are dropped (they must be
    rebuilt from the vertices); vertex coordinates are unchanged."""
    rots = cube_rotations()
    choice = _rng(seed).integers(0, len(rots), size=mesh["E"])
    corners = np.array([[v & 1, (v >> 1) & 1, (v >> 2) & 1] for v in range(8)], dtype=np.int64)
    maps = []
    for R in rots:
        old = ((R @ (2 * corners.T - 1)) + 1) // 2            # [3, 8]
        maps.append(old[0] + 2 * old[1] + 4 * old[2])
    maps = np.array(maps)                                      # [24, 8]
    ev = mesh["elem_verts"]
    new_ev = np.take_along_axis(ev, maps[choice], axis=1).astype(np.int32)
    return dict(vert_xyz=mesh["vert_xyz"], elem_verts=np.ascontiguousarray(new_ev), p=mesh["p"],
                E=mesh["E"], n=mesh.get("n"))


def elements_of_nodes(mesh, rows):
    """CSR list of the elements that contain each global node in `rows`.

    Pure index arithmetic on the structured lattice: node (I,J,K) lies in the
    elements (ex,ey,ez) with p*ex <= I <= p*ex + p.  Returns (row_ptr, elems),
    element ids in the (possibly shuffled) order of mesh['elem_nodes'].
    """
    n, p, M = mesh["n"], mesh["p"], mesh["M"]
    inv = np.empty_like(mesh["perm"])
    inv[mesh["perm"]] = np.arange(mesh["perm"].size)
    rows = np.asarray(rows, dtype=np.int64)
    I = rows % M
    J = (rows // M) % M
    K = rows // (M * M)
    ptr = [0]
    out = []
    for a, b, c in zip(I, J, K):
        def rng1(t):
            lo = max(0, -(-(t - p) // p))
            hi = min(n - 1, t // p)
            return range(lo, hi + 1)
        for ez in rng1(c):
            for ey in rng1(b):
                for ex in rng1(a):
                    out.append(inv[ex + n * (ey + n * ez)])
        ptr.append(len(out))
    return np.asarray(ptr, dtype=np.int64), np.asarray(out, dtype=np.int64)


def rhs_uniform(N, dirichlet=None, seed=0, ncomp=1):
    """b ~ U[-1, 1] per component, zero on Dirichlet nodes; [ncomp*N] float64."""
    b = _rng(seed).uniform(-1.0, 1.0, size=(ncomp, N))
    if dirichlet is not None:
        b[:, dirichlet.astype(bool)] = 0.0
    return np.ascontiguousarray(b.reshape(-1))


def rff_params(M=1024, ell=0.1, seed=0):
    """Random Fourier feature draws for a squared-exponential field of
    correlation length ell: [M, 4] = (w_x, w_y, w_z, b), w ~ N(0, ell^-2 I),
    b ~ U[0, 2 pi)."""
    rng = _rng(seed)
    w = rng.normal(0.0, 1.0 / ell, size=(M, 3))
    b = rng.uniform(0.0, 2.0 * np.pi, size=(M, 1))
    return np.ascontiguousarray(np.concatenate([w, b], axis=1))


def bp3_mesh_n(target_dofs, p):
    """Elements per direction for a BP3 sweep point: round((N_t^(1/3) - 1)/p)."""
    return max(1, int(round((target_dofs ** (1.0 / 3.0) - 1.0) / p)))


def batch_problems(count=64, seed=7, nmin=4, nmax=32, pmin=2, pmax=8):
    """The batched workload: `count` independent BP3 problems with n in
    [nmin, nmax] elements per direction and p in [pmin, pmax], drawn from a seed.
    Returns a list of dicts (n, p, mesh_seed, rhs_seed)."""
    rng = _rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    ps = rng.integers(pmin, pmax + 1, size=count)
    return [dict(n=int(ns[k]), p=int(ps[k]), mesh_seed=1000 + k, rhs_seed=2000 + k)
            for k in range(count)]


def mlp_init(n_in, n_h, n_out, seed=0, out_scale=0.1):
    """Initial weights of the per-element perceptron: He-uniform draws
    U(-sqrt(6/fan_in), sqrt(6/fan_in)) (the last layer scaled by out_scale),
    zero biases; flat float32 array in the order W1, b1, W2, b2, W3, b3."""
    rng = _rng(seed)
    parts = []
    for fan_in, fan_out, sc in ((n_in, n_h, 1.0), (n_h, n_h, 1.0), (n_h, n_out, out_scale)):
        lim = np.sqrt(6.0 / fan_in) * sc
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)

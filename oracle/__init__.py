"""FP64 CPU oracle for the CEED bake-off operators (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
import this package.  It shares no code with the CUDA library
(paper_2109_04996_b300); both consume the arrays of `fem_inputs`.

What it computes, and where the paper defines it (Kolev et al. 2021):
  * 1D Gauss-Legendre (q = p+2, BP1-BP4) and Gauss-Lobatto-Legendre
    (q = p+1, BP5/BP6) rules                        -- section "Benchmarks"
  * isoparametric Q_p bricks x^e(r), r in [-1,1]^3   -- section "Benchmarks"
  * A_ij = int grad phi_i . grad phi_j, B_ij = int phi_i phi_j, by brute-force
    tensor quadrature with dense 3D basis tables     -- section "Benchmarks"
  * y = sum_e G_e^T K_e G_e x                         -- section "libCEED"
  * CG with a diagonal (Jacobi) preconditioner        -- section "Miniapps"
    (Nekbone) and section "Benchmarks" (CG on the BP systems)
The brute-force C code is oracle/oracle.c; this file adds numpy-level helpers
(assembled matrices for tiny meshes, the CG loops) that call it.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MASS, DIFFUSION = 0, 1
GAUSS, LOBATTO = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_int64)
        L.oracle_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.oracle_gauss_lobatto.argtypes = [ctypes.c_int, dp, dp]
        L.oracle_lagrange_1d.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.oracle_nodes_from_vertices.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ip, ip, dp]
        L.oracle_op_new.restype = ctypes.c_void_p
        L.oracle_op_new.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ip, dp,
                                    ctypes.c_int, ctypes.c_double, dp]
        L.oracle_op_free.argtypes = [ctypes.c_void_p]
        L.oracle_qdata.argtypes = [ctypes.c_void_p, ctypes.c_int64, dp]
        L.oracle_element_matrix.argtypes = [ctypes.c_void_p, ctypes.c_int64, dp]
        L.oracle_apply.argtypes = [ctypes.c_void_p, dp, dp, ip, ctypes.c_int64, ctypes.c_int]
        L.oracle_apply_rows.argtypes = [ctypes.c_void_p, dp, ctypes.c_int64, lp, lp, lp, dp,
                                        ctypes.c_int]
        L.oracle_diagonal.argtypes = [ctypes.c_void_p, dp]
        L.oracle_rhs.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        L.oracle_error_norms.argtypes = [ctypes.c_void_p, dp, dp]
        L.oracle_quadrature_points.argtypes = [ctypes.c_void_p, ctypes.c_int64, dp]
        L.oracle_kappa.restype = ctypes.c_double
        L.oracle_kappa.argtypes = [ctypes.c_void_p, dp]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_mlp_nparams.restype = ctypes.c_int64
        L.oracle_mlp_nparams.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_mlp_forward.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                         ctypes.c_int, dp, dp, dp, dp]
        L.oracle_mlp_loss_grad.restype = ctypes.c_double
        L.oracle_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                           ctypes.c_int, dp, dp, dp]
        L.oracle_adam_step.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def gauss_legendre(q):
    x = np.zeros(q); w = np.zeros(q)
    if lib().oracle_gauss_legendre(q, _dp(x), _dp(w)):
        raise ValueError(q)
    return x, w


def gauss_lobatto(P):
    x = np.zeros(P); w = np.zeros(P)
    if lib().oracle_gauss_lobatto(P, _dp(x), _dp(w)):
        raise ValueError(P)
    return x, w


def lagrange_1d(p, r):
    """Values and derivatives of the Gauss-Lobatto Lagrange basis of order p at
    the points r: two [len(r), p+1] arrays."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    v = np.zeros((r.size, p + 1)); d = np.zeros((r.size, p + 1))
    lib().oracle_lagrange_1d(p, r.size, _dp(r), _dp(v), _dp(d))
    return v, d


def nodes_from_vertices(mesh):
    """Coordinates [N, 3] of the Q_p nodes of the trilinear bricks of `mesh`."""
    xyz = np.zeros((mesh["N"], 3))
    ev = np.ascontiguousarray(mesh["elem_verts"], dtype=np.int32)
    en = np.ascontiguousarray(mesh["elem_nodes"], dtype=np.int32)
    vx = np.ascontiguousarray(mesh["vert_xyz"], dtype=np.float64)
    lib().oracle_nodes_from_vertices(mesh["p"], mesh["E"], _dp(vx), _ip(ev), _ip(en), _dp(xyz))
    return xyz


class Operator:
    """Oracle for one operator (mass or diffusion) on one Q_p mesh.

    kind: MASS or DIFFUSION; quad: GAUSS (q points) or LOBATTO (q = p+1);
    ncomp: 1 or 3; rff: None or the [M, 4] random-feature draws of kappa(x).
    """

    def __init__(self, mesh, kind, quad, q, ncomp=1, node_xyz=None, rff=None, sigma=1.0,
                 nthreads=0):
        self.mesh = mesh
        self.p = mesh["p"]; self.P = self.p + 1
        self.N = mesh["N"]; self.E = mesh["E"]
        self.kind, self.quad, self.q, self.ncomp = kind, quad, q, ncomp
        self.nthreads = nthreads
        self.elem_nodes = np.ascontiguousarray(mesh["elem_nodes"], dtype=np.int32)
        self.node_xyz = np.ascontiguousarray(
            nodes_from_vertices(mesh) if node_xyz is None else node_xyz, dtype=np.float64)
        M = 0
        self.rff = None
        if rff is not None:
            self.rff = np.ascontiguousarray(rff, dtype=np.float64)
            M = self.rff.shape[0]
        self.sigma = float(sigma)
        self._h = lib().oracle_op_new(self.p, q, quad, kind, ncomp, self.N, self.E,
                                      _ip(self.elem_nodes), _dp(self.node_xyz), M, self.sigma,
                                      _dp(self.rff) if self.rff is not None else None)
        if not self._h:
            raise ValueError("invalid oracle operator parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_op_free(h)
            self._h = None

    @property
    def nq(self):
        return self.q ** 3

    def apply(self, x, elems=None):
        """y = sum_e G_e^T K_e G_e x (all elements, or the listed ones)."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        assert x.size == self.ncomp * self.N
        y = np.zeros_like(x)
        if elems is None:
            rc = lib().oracle_apply(self._h, _dp(x), _dp(y), None, 0, self.nthreads)
        else:
            el = np.ascontiguousarray(elems, dtype=np.int32)
            rc = lib().oracle_apply(self._h, _dp(x), _dp(y), _ip(el), el.size, self.nthreads)
        if rc:
            raise ValueError("element index out of range")
        return y

    def apply_rows(self, x, rows, row_ptr, row_elems):
        """Entries y[rows] of the full product, from the elements listed per row."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        re = np.ascontiguousarray(row_elems, dtype=np.int64)
        out = np.zeros(rows.size)
        if lib().oracle_apply_rows(self._h, _dp(x), rows.size, _lp(rows), _lp(rp), _lp(re),
                                   _dp(out), self.nthreads):
            raise ValueError("bad rows")
        return out

    def element_matrix(self, e):
        K = np.zeros((self.P ** 3, self.P ** 3))
        if lib().oracle_element_matrix(self._h, e, _dp(K)):
            raise IndexError(e)
        return K

    def qdata(self, e):
        nd = 1 if self.kind == MASS else 6
        out = np.zeros(nd * self.nq)
        if lib().oracle_qdata(self._h, e, _dp(out)):
            raise IndexError(e)
        return out.reshape(nd, self.nq)

    def quadrature_points(self, e):
        out = np.zeros((self.nq, 3))
        lib().oracle_quadrature_points(self._h, e, _dp(out))
        return out

    def kappa(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return lib().oracle_kappa(self._h, _dp(x))

    def diagonal(self):
        d = np.zeros(self.N)
        lib().oracle_diagonal(self._h, _dp(d))
        return np.tile(d, self.ncomp)

    def rhs(self, which):
        """b_i = int phi_i f, f = sin sin sin (which=0) or 3 pi^2 sin sin sin (1)."""
        b = np.zeros(self.N)
        lib().oracle_rhs(self._h, which, _dp(b))
        return b

    def error_norms(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(2)
        lib().oracle_error_norms(self._h, _dp(u), _dp(out))
        return out

    def assembled(self):
        """Dense N x N scalar matrix sum_e G_e^T K_e G_e (tiny meshes only)."""
        N = self.N
        if N > 6000:
            raise ValueError("assembled() is for tiny meshes")
        A = np.zeros((N, N))
        for e in range(self.E):
            g = self.elem_nodes[e]
            A[np.ix_(g, g)] += self.element_matrix(e)
        return A


def constrained(y, x, dirichlet, ncomp=1):
    """Dirichlet form of a product (paper: homogeneous Dirichlet on all BPs):
    A_c x = M A M x + (I - M) x with M the interior mask.  `y` must be A (M x)."""
    m = np.tile(dirichlet.astype(bool), ncomp)
    out = y.copy()
    out[m] = x[m]
    return out


def pcg(op, b, dirichlet, rtol=1e-10, maxit=10000, precond="jacobi", x0=None):
    """Preconditioned conjugate gradients on the Dirichlet-constrained system,
    in plain FP64 numpy around the brute-force apply.

    The system is A_c x = b with A_c = M A M + (I - M); b must vanish on the
    Dirichlet nodes, so does every iterate.  precond: "none" or "jacobi"
    (z = r / diag(A) on interior nodes).  Stops when ||r||_2 <= rtol ||b||_2 or
    after maxit iterations.  Returns (x, iterations, ||r||/||b|| history).
    """
    nc = op.ncomp
    m = np.tile(dirichlet.astype(bool), nc)
    inner = ~m
    b = np.where(inner, b, 0.0)
    x = np.zeros_like(b) if x0 is None else np.where(inner, x0, 0.0)

    def A(v):
        return np.where(inner, op.apply(v), 0.0)

    dinv = None
    if precond == "jacobi":
        d = op.diagonal()
        dinv = np.where(inner, 1.0 / np.where(inner, d, 1.0), 0.0)
    r = b - A(x)
    z = r * dinv if dinv is not None else r.copy()
    p = z.copy()
    rz = r @ z
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0]
    k = 0
    while k < maxit and hist[-1] > rtol:
        Ap = A(p)
        pAp = p @ Ap
        alpha = rz / pAp
        x += alpha * p
        r -= alpha * Ap
        z = r * dinv if dinv is not None else r.copy()
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        k += 1
        hist.append(np.linalg.norm(r) / bnorm)
    return x, k, np.asarray(hist)


def max_threads():
    return lib().oracle_max_threads()


# ---------------------------------------------------------------- MLP (oracle/mlp.c)

def mlp_nparams(n_in, n_h, n_out):
    return lib().oracle_mlp_nparams(n_in, n_h, n_out)


def mlp_forward(dims, params, x):
    """FP64 forward of the 3-layer ReLU perceptron; returns (y, h1, h2)."""
    n_in, n_h, n_out = dims
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    S = x.shape[0]
    y = np.zeros((S, n_out)); h1 = np.zeros((S, n_h)); h2 = np.zeros((S, n_h))
    lib().oracle_mlp_forward(n_in, n_h, n_out, _dp(p), S, _dp(x), _dp(y), _dp(h1), _dp(h2))
    return y, h1, h2


def mlp_loss_grad(dims, params, x, t):
    """L = mean over rows of ||y - t||^2 and dL/dparams (FP64)."""
    n_in, n_h, n_out = dims
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    g = np.zeros_like(p)
    L = lib().oracle_mlp_loss_grad(n_in, n_h, n_out, _dp(p), x.shape[0], _dp(x), _dp(t), _dp(g))
    return L, g


def adam_step(params, grad, m, v, k, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step k (>= 1) on FP64 arrays."""
    lib().oracle_adam_step(params.size, _dp(params), _dp(np.ascontiguousarray(grad)), _dp(m),
                           _dp(v), k, lr, b1, b2, eps)

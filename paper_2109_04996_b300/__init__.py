"""B300-native matrix-free high-order finite element operators (CEED bake-off
problems BP1-BP6, Kolev et al., sections "Benchmarks" and "libCEED").

A thin ctypes binding over libfem.so (C ABI declared in include/fem.h):
argument marshalling only; every step of the operator and the solvers runs in
the library's CUDA kernels.  PyTorch provides device memory and the stream.
The library must be built (``python -m paper_2109_04996_b300.build``); there
is no fallback when it is missing.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libfem.so")

MASS, DIFFUSION = 0, 1
GAUSS, LOBATTO = 0, 1
F64, F32 = 0, 1
PC_NONE, PC_JACOBI, PC_LEARNED = 0, 1, 2
STATUS = {0: "FEM_OK", 1: "FEM_EINVAL", 2: "FEM_ENOMEM", 3: "FEM_ECUDA", 4: "FEM_EBREAKDOWN",
          5: "FEM_ENOCONV", 6: "FEM_ETIMEOUT", 7: "FEM_EDEVICE"}

# The bake-off problems (section "Benchmarks"): kind, components, quadrature, q - p.
BAKE_OFF = {
    "BP1": (MASS, 1, GAUSS, 2), "BP2": (MASS, 3, GAUSS, 2),
    "BP3": (DIFFUSION, 1, GAUSS, 2), "BP4": (DIFFUSION, 3, GAUSS, 2),
    "BP5": (DIFFUSION, 1, LOBATTO, 1), "BP6": (DIFFUSION, 3, LOBATTO, 1),
}


class FemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class _TuneResult(ctypes.Structure):
    _fields_ = [("epb_choice", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("us", ctypes.c_double), ("from_cache", ctypes.c_int),
                ("candidates", ctypes.c_int)]


class _CgOpts(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int), ("maxit", ctypes.c_int), ("rtol", ctypes.c_double),
                ("use_graph", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("zero_guess", ctypes.c_int)]


class _CgStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("status", ctypes.c_int),
                ("rnorm", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("true_rel", ctypes.c_double), ("fallback", ctypes.c_int)]


_lib = None
_VP = ctypes.c_void_p

# fem_comm callbacks of fem_pcg_dist
_CommSum = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_CommReduce = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                               ctypes.c_int)


class _Comm(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("sum_interfaces", _CommSum),
                ("allreduce", _CommReduce)]
_I64 = ctypes.c_int64


class _PmgOpts(ctypes.Structure):
    _fields_ = [("cheb_degree", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("power_its", ctypes.c_int),
                ("coarse_its", ctypes.c_int), ("prec", ctypes.c_int)]


def lib():
    """Load libfem.so.  Raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise ImportError("libfem.so not built: run `python -m paper_2109_04996_b300.build`")
    L = ctypes.CDLL(LIBPATH)
    L.fem_last_error.restype = ctypes.c_char_p
    sigs = {
        "fem_basis_tables": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP, _VP],
        "fem_mesh_nodes_from_vertices": [ctypes.c_int, _I64, _I64, _VP, _VP, _VP, _I64, _VP],
        "fem_mesh_create": [ctypes.c_int, _I64, _I64, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)],
        "fem_mesh_destroy": [_VP],
        "fem_mesh_create_vertices": [ctypes.c_int, _I64, _I64, _VP, _I64, _VP, _VP, _VP, _VP,
                                     ctypes.POINTER(_VP)],
        "fem_mesh_node_coords": [_VP, _VP],
        "fem_mesh_box": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                         ctypes.c_uint64, _VP, ctypes.POINTER(_VP)],
        "fem_mesh_connectivity": [ctypes.c_int, _I64, _I64, _VP, _VP, _VP,
                                  ctypes.POINTER(ctypes.c_int64)],
        "fem_op_create": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_int, _VP, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_VP)],
        "fem_op_destroy": [_VP],
        "fem_op_sizes": [_VP, _VP, _VP, _VP, _VP, _VP, _VP],
        "fem_op_apply": [_VP, _VP, _VP],
        "fem_op_apply_f32": [_VP, _VP, _VP],
        "fem_op_apply_elements": [_VP, _VP, _I64, _VP, _VP],
        "fem_op_diagonal": [_VP, _VP],
        "fem_op_qdata_host": [_VP, _I64, _VP],
        "fem_op_rhs": [_VP, ctypes.c_int, _VP],
        "fem_cg_solve": [_VP, _VP, _VP, ctypes.POINTER(_CgOpts), ctypes.POINTER(_CgStats)],
        "fem_solve_refined": [_VP, _VP, _VP, ctypes.POINTER(_CgOpts), ctypes.POINTER(_CgStats)],
        "fem_pcg_dist": [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_CgOpts), ctypes.POINTER(_Comm),
                         ctypes.POINTER(_CgStats)],
        "fem_cg_checkpoint_size": [_VP, ctypes.POINTER(ctypes.c_int64)],
        "fem_cg_checkpoint": [_VP, _VP],
        "fem_cg_restore": [_VP, _VP],
        "fem_cg_resume": [_VP, _VP, _VP, ctypes.POINTER(_CgOpts), ctypes.POINTER(_CgStats)],
        "fem_op_set_launch_shape": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int],
        "fem_op_autotune": [_VP, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(_TuneResult)],
        "fem_op_residual": [_VP, _VP, _VP, _VP],
        "fem_mlp_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP,
                           ctypes.POINTER(_VP)],
        "fem_mlp_destroy": [_VP],
        "fem_mlp_save": [_VP, ctypes.c_char_p],
        "fem_mlp_load": [ctypes.c_char_p, _VP, ctypes.POINTER(_VP)],
        "fem_mlp_params": [_VP, _VP, ctypes.POINTER(ctypes.c_int64)],
        "fem_mlp_forward": [_VP, _VP, _I64, _VP],
        "fem_mlp_train_step": [_VP, _VP, _VP, _I64, ctypes.c_int, ctypes.c_float, _VP,
                               ctypes.POINTER(ctypes.c_double)],
        "fem_mlp_train": [_VP, _VP, _VP, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                          ctypes.c_float, ctypes.c_uint64, _VP],
        "fem_mlp_train_plateau": [_VP, _VP, _VP, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_float, ctypes.c_uint64,
                                  _VP, ctypes.POINTER(ctypes.c_int)],
        "fem_precond_create": [_VP, _VP, ctypes.POINTER(_VP)],
        "fem_precond_create_pmg": [_VP, ctypes.POINTER(_VP)],
        "fem_precond_destroy": [_VP],
        "fem_precond_features": [_VP, _VP],
        "fem_precond_samples": [_VP, _VP, _VP, _VP, _VP, _VP],
        "fem_precond_apply": [_VP, _VP, _VP],
        "fem_precond_set_gamma": [_VP, ctypes.c_double],
        "fem_precond_calibrate": [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_double)],
        "fem_fcg_solve": [_VP, _VP, _VP, ctypes.POINTER(_CgOpts), ctypes.POINTER(_CgStats)],
        "fem_batch_create": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)],
        "fem_batch_create_split": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int64,
                                   ctypes.POINTER(_VP)],
        "fem_batch_graph_state": [_VP, ctypes.POINTER(ctypes.c_int)],
        "fem_batch_destroy": [_VP],
        "fem_batch_solve": [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                            ctypes.POINTER(_CgOpts), ctypes.POINTER(_CgStats)],
        "fem_batch_set_shape": [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double],
        "fem_batch_autotune": [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int,
                               ctypes.POINTER(_TuneResult)],
        "fem_batch_barrier_selftest": [_VP, ctypes.c_double],
        "fem_pmg_create": [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_PmgOpts),
                           ctypes.POINTER(_VP)],
        "fem_pmg_destroy": [_VP],
        "fem_pmg_get_lmax": [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
        "fem_pmg_set_lmax": [_VP, ctypes.c_int, ctypes.c_double],
        "fem_pmg_prolong": [_VP, ctypes.c_int, _VP, _VP],
        "fem_pmg_restrict": [_VP, ctypes.c_int, _VP, _VP],
        "fem_pmg_vcycle": [_VP, _VP, _VP],
        "fem_pmg_solve": [_VP, _VP, _VP, ctypes.POINTER(_CgOpts), ctypes.POINTER(_CgStats)],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise FemError(rc, lib().fem_last_error().decode())


def _ptr(t):
    """Device pointer of a CUDA tensor (or host pointer of a numpy array)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _vec(t, dtype, n, what="vector"):
    """Device pointer of a contiguous CUDA tensor of `n` elements of `dtype`
    (the library reads and writes exactly that many; anything else would
    make it touch memory outside the tensor)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (what, dtype, t.dtype))
    if t.numel() != n:
        raise ValueError("%s must have %d elements, got %d" % (what, n, t.numel()))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def basis_tables(p, q, quad):
    P = p + 1
    out = [np.zeros(P), np.zeros(q), np.zeros(q), np.zeros((q, P)), np.zeros((q, P))]
    _check(lib().fem_basis_tables(p, q, quad, *[_ptr(a) for a in out]))
    return dict(nodes=out[0], qpts=out[1], qwts=out[2], interp=out[3], grad=out[4])


def mesh_connectivity(p, vert_xyz, elem_verts):
    """Q_p connectivity of a hexahedral mesh given by its vertices
    (fem_mesh_connectivity, host): returns a mesh dict like
    fem_inputs.box_mesh's (vert_xyz, elem_verts, elem_nodes, dirichlet, n=None,
    p, N, E), with Dirichlet nodes on the faces of one element only."""
    ev = np.ascontiguousarray(elem_verts, dtype=np.int32)
    vx = np.ascontiguousarray(vert_xyz, dtype=np.float64)
    E = ev.shape[0]
    P = p + 1
    en = np.empty((E, P ** 3), dtype=np.int32)
    dr = np.empty(E * P ** 3, dtype=np.uint8)
    N = ctypes.c_int64()
    _check(lib().fem_mesh_connectivity(int(p), vx.shape[0], E, ev.ctypes.data, en.ctypes.data,
                                       dr.ctypes.data, ctypes.byref(N)))
    N = N.value
    return dict(vert_xyz=vx, elem_verts=ev, elem_nodes=en, dirichlet=dr[:N].copy(), n=None,
                p=int(p), N=N, E=E, M=None, perm=np.arange(E, dtype=np.int64))


def nodes_from_vertices(mesh):
    """Q_p node coordinates [N, 3] of the trilinear bricks of a mesh dict."""
    xyz = np.zeros((mesh["N"], 3))
    vx = np.ascontiguousarray(mesh["vert_xyz"], dtype=np.float64)
    ev = np.ascontiguousarray(mesh["elem_verts"], dtype=np.int32)
    en = np.ascontiguousarray(mesh["elem_nodes"], dtype=np.int32)
    _check(lib().fem_mesh_nodes_from_vertices(mesh["p"], mesh["E"], vx.shape[0], _ptr(vx),
                                               _ptr(ev), _ptr(en), mesh["N"], _ptr(xyz)))
    return xyz


class Mesh:
    """A Q_p hexahedral mesh resident on the GPU (elem_nodes, coordinates,
    Dirichlet marker).  `mesh` is a dict as produced by fem_inputs.box_mesh;
    node coordinates come from the library's own trilinear map unless given."""

    def __init__(self, mesh, node_xyz=None, stream=None):
        self.p = int(mesh["p"]); self.N = int(mesh["N"]); self.E = int(mesh["E"])
        P3 = (self.p + 1) ** 3
        en = np.ascontiguousarray(mesh["elem_nodes"], dtype=np.int32)
        if en.size != self.E * P3:
            raise ValueError("elem_nodes must hold E * (p+1)^3 = %d ids, got %d" % (self.E * P3, en.size))
        dr = mesh.get("dirichlet")
        dr = None if dr is None else np.ascontiguousarray(dr, dtype=np.uint8)
        if dr is not None and dr.size != self.N:
            raise ValueError("dirichlet must have N = %d entries, got %d" % (self.N, dr.size))
        if node_xyz is None:
            ev = np.asarray(mesh["elem_verts"])
            if ev.shape != (self.E, 8) or np.asarray(mesh["vert_xyz"]).shape[1:] != (3,):
                raise ValueError("elem_verts must be [E, 8] and vert_xyz [nvert, 3]")
        elif np.asarray(node_xyz).size != 3 * self.N:
            raise ValueError("node_xyz must be [N, 3]")
        self.dirichlet = dr
        h = _VP()
        if node_xyz is None:
            # node coordinates computed on the GPU from the trilinear bricks
            vx = np.ascontiguousarray(mesh["vert_xyz"], dtype=np.float64)
            ev = np.ascontiguousarray(mesh["elem_verts"], dtype=np.int32)
            _check(lib().fem_mesh_create_vertices(self.p, self.N, self.E, _ptr(en), vx.shape[0],
                                                  _ptr(vx), _ptr(ev), _ptr(dr),
                                                  _stream_handle(stream), ctypes.byref(h)))
            self._xyz = None
        else:
            self._xyz = np.ascontiguousarray(node_xyz, dtype=np.float64)
            _check(lib().fem_mesh_create(self.p, self.N, self.E, _ptr(en), _ptr(self._xyz),
                                         _ptr(dr), _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    @classmethod
    def box(cls, p, nx, ny=None, nz=None, perturb=0.1, seed=0, stream=None):
        """The library's bake-off mesh generator (fem_mesh_box): nx*ny*nz
        perturbed bricks of the unit cube with Q_p nodes, built and uploaded
        by the library."""
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        h = _VP()
        _check(lib().fem_mesh_box(int(p), int(nx), int(ny), int(nz), float(perturb), int(seed),
                                  _stream_handle(stream), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.p = int(p)
        self.E = int(nx) * int(ny) * int(nz)
        self.N = (p * nx + 1) * (p * ny + 1) * (p * nz + 1)
        self.dirichlet = None
        self._xyz = None
        self._h = h
        return self

    @property
    def node_xyz(self):
        """Node coordinates [N, 3] (copied from the device on first use)."""
        if self._xyz is None:
            xyz = np.zeros((self.N, 3))
            _check(lib().fem_mesh_node_coords(self._h, _ptr(xyz)))
            self._xyz = xyz
        return self._xyz

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fem_mesh_destroy(self._h)
            self._h = None


class Operator:
    """y = G^T B^T D B G x on a Mesh (see include/fem.h, fem_op_create)."""

    def __init__(self, mesh, kind, quad, q, ncomp=1, prec=F64, rff=None, sigma=1.0):
        self.mesh = mesh
        self.kind, self.quad, self.q, self.ncomp, self.prec = kind, quad, q, ncomp, prec
        self.N, self.E, self.p = mesh.N, mesh.E, mesh.p
        rff_a = None if rff is None else np.ascontiguousarray(rff, dtype=np.float64)
        M = 0 if rff_a is None else rff_a.shape[0]
        h = _VP()
        _check(lib().fem_op_create(mesh._h, kind, quad, q, ncomp, prec, _ptr(rff_a), M,
                                   float(sigma), ctypes.byref(h)))
        self._h = h

    @classmethod
    def bake_off(cls, mesh, name, prec=F64, **kw):
        kind, ncomp, quad, dq = BAKE_OFF[name]
        return cls(mesh, kind, quad, mesh.p + dq, ncomp=ncomp, prec=prec, **kw)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fem_op_destroy(self._h)
            self._h = None

    @property
    def n(self):
        return self.ncomp * self.N

    def device_bytes(self):
        b = ctypes.c_int64()
        _check(lib().fem_op_sizes(self._h, None, None, None, None, None, ctypes.byref(b)))
        return b.value

    def apply(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(lib().fem_op_apply(self._h, _vec(x, torch.float64, self.n, "x"),
                                  _vec(y, torch.float64, self.n, "y")))
        return y

    def apply_f32(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(lib().fem_op_apply_f32(self._h, _vec(x, torch.float32, self.n, "x"),
                                      _vec(y, torch.float32, self.n, "y")))
        return y

    def apply_elements(self, elems, x, y=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(lib().fem_op_apply_elements(self._h, _vec(elems, torch.int32, elems.numel(), "elems"),
                                           elems.numel(), _vec(x, torch.float64, self.n, "x"),
                                           _vec(y, torch.float64, self.n, "y")))
        return y

    def diagonal(self, d=None):
        import torch
        if d is None:
            d = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(lib().fem_op_diagonal(self._h, _vec(d, torch.float64, self.n, "d")))
        return d

    def qdata(self, e):
        nd = 6 if self.kind == DIFFUSION else 1
        out = np.zeros((nd, self.q ** 3))
        _check(lib().fem_op_qdata_host(self._h, e, _ptr(out)))
        return out

    def rhs(self, which, b=None):
        import torch
        if b is None:
            b = torch.empty(self.N, dtype=torch.float64, device="cuda")
        _check(lib().fem_op_rhs(self._h, which, _vec(b, torch.float64, self.N, "b")))
        return b

    def cg(self, b, x, precond=PC_JACOBI, maxit=10000, rtol=1e-10, use_graph=True,
           zero_guess=False):
        """Solve the Dirichlet-constrained system in place (x: initial guess
        in, solution out; zero_guess=True starts from 0 whatever x holds and
        skips the initial residual's apply).  Returns the statistics as a
        dict; raises FemError on breakdown, returns status FEM_ENOCONV without
        raising."""
        o = _CgOpts(precond, int(maxit), float(rtol), 1 if use_graph else 0, 0.0, 0,
                    1 if zero_guess else 0)
        st = _CgStats()
        import torch
        rc = lib().fem_cg_solve(self._h, _vec(b, torch.float64, self.n, "b"),
                                _vec(x, torch.float64, self.n, "x"), ctypes.byref(o), ctypes.byref(st))
        if rc not in (0, 5):
            _check(rc)
        return _stats(st)

    def cg_checkpoint(self):
        """The state of this operator's last CG solve (fem_cg_checkpoint) as
        a host byte array."""
        n = ctypes.c_int64()
        _check(lib().fem_cg_checkpoint_size(self._h, ctypes.byref(n)))
        buf = np.zeros(n.value, dtype=np.uint8)
        _check(lib().fem_cg_checkpoint(self._h, _ptr(buf)))
        return buf

    def cg_restore(self, state):
        """Load a state from cg_checkpoint (fem_cg_restore)."""
        buf = np.ascontiguousarray(state, dtype=np.uint8)
        _check(lib().fem_cg_restore(self._h, _ptr(buf)))

    def cg_resume(self, b, x, precond=PC_JACOBI, maxit=10000, rtol=1e-10):
        """Continue an interrupted solve from x (fem_cg_resume)."""
        import torch
        o = _CgOpts(precond, int(maxit), float(rtol), 0, 0.0, 0, 0)
        st = _CgStats()
        rc = lib().fem_cg_resume(self._h, _vec(b, torch.float64, self.n, "b"),
                                 _vec(x, torch.float64, self.n, "x"), ctypes.byref(o), ctypes.byref(st))
        if rc not in (0, 5):
            _check(rc)
        return _stats(st)

    def residual(self, b, x, r=None):
        """r = M (b - A x) in FP64 (Dirichlet entries 0)."""
        import torch
        if r is None:
            r = torch.empty_like(x)
        _check(lib().fem_op_residual(self._h, _vec(b, torch.float64, self.n, "b"),
                                     _vec(x, torch.float64, self.n, "x"),
                                     _vec(r, torch.float64, self.n, "r")))
        return r

    def set_launch_shape(self, prec, epb_choice, blocks_per_sm=0):
        _check(lib().fem_op_set_launch_shape(self._h, prec, epb_choice, blocks_per_sm))

    def autotune(self, prec=F64, cache=None):
        """Time the apply's launch shapes and keep the fastest (see
        fem_op_autotune).  Returns the chosen shape as a dict."""
        r = _TuneResult()
        _check(lib().fem_op_autotune(self._h, prec, None if cache is None else cache.encode(),
                                     ctypes.byref(r)))
        return dict(epb_choice=r.epb_choice, blocks_per_sm=r.blocks_per_sm, us=r.us,
                    from_cache=bool(r.from_cache), candidates=r.candidates)

    def solve_refined(self, b, x, rtol=1e-10, inner_rtol=0.1, maxit=100000, max_outer=100,
                      precond=PC_JACOBI):
        """FP64 iterative refinement around an FP32 inner PCG (operator
        created with prec=F32).  x: initial guess in, solution out."""
        o = _CgOpts(precond, int(maxit), float(rtol), 1, float(inner_rtol), int(max_outer))
        st = _CgStats()
        import torch
        rc = lib().fem_solve_refined(self._h, _vec(b, torch.float64, self.n, "b"),
                                     _vec(x, torch.float64, self.n, "x"), ctypes.byref(o),
                                     ctypes.byref(st))
        if rc not in (0, 5):
            _check(rc)
        return _stats(st)


def _stats(st):
    return dict(iterations=st.iterations, outer=st.outer, status=STATUS[st.status],
                rnorm=st.rnorm, bnorm=st.bnorm, true_rel=st.true_rel, fallback=st.fallback)


class Batch:
    """Independent BP3/BP4-type problems (FP32 operators, Gauss q = p+2)
    solved together: FP64 refinement, the inner FP32 PCG of all problems in
    one persistent kernel per outer step (include/fem.h, fem_batch_*)."""

    SOLO_DOFS = 1 << 21   # FEM_BATCH_SOLO_DOFS

    def __init__(self, ops, solo_dofs=None):
        """solo_dofs: problems with at least this many unknowns are solved
        one after another with their own refined solve instead of in the
        persistent kernel (None: the library default, <= 0: never)."""
        self.ops = list(ops)
        self.solo_dofs = self.SOLO_DOFS if solo_dofs is None else int(solo_dofs)
        arr = (_VP * len(self.ops))(*[o._h for o in self.ops])
        h = _VP()
        _check(lib().fem_batch_create_split(arr, len(self.ops), self.solo_dofs, ctypes.byref(h)))
        self._h = h

    @property
    def solo(self):
        """Indices of the problems solved alone."""
        if self.solo_dofs <= 0:
            return []
        return [i for i, o in enumerate(self.ops) if o.n >= self.solo_dofs]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fem_batch_destroy(self._h)
            self._h = None

    def _vecs(self, bs, xs):
        import torch
        if not (len(bs) == len(self.ops) == len(xs)):
            raise ValueError("one right-hand side and one solution per problem")
        bp = [_vec(b, torch.float64, op.n, "b") for b, op in zip(bs, self.ops)]
        xp = [_vec(x, torch.float64, op.n, "x") for x, op in zip(xs, self.ops)]
        return (_VP * len(bs))(*bp), (_VP * len(xs))(*xp)

    def solve(self, bs, xs, rtol=1e-10, inner_rtol=0.1, maxit=100000, max_outer=100):
        o = _CgOpts(PC_JACOBI, int(maxit), float(rtol), 0, float(inner_rtol), int(max_outer))
        st = (_CgStats * len(self.ops))()
        bv, xv = self._vecs(bs, xs)
        rc = lib().fem_batch_solve(self._h, bv, xv, ctypes.byref(o), st)
        if rc not in (0, 5):
            _check(rc)
        return [_stats(s) for s in st]

    def set_shape(self, nt_choice, blocks_per_sm=0, timeout_ms=2000.0):
        _check(lib().fem_batch_set_shape(self._h, nt_choice, blocks_per_sm, timeout_ms))

    def autotune(self, bs, xs, iters=10):
        r = _TuneResult()
        bv, xv = self._vecs(bs, xs)
        _check(lib().fem_batch_autotune(self._h, bv, xv, iters, ctypes.byref(r)))
        return dict(nt_choice=r.epb_choice, blocks_per_sm=r.blocks_per_sm, us_per_iter=r.us,
                    candidates=r.candidates)

    def graph_state(self):
        """1: the refinement loop runs as one CUDA graph; 0: not captured yet;
        -1: capture refused, host-launched steps (fem_batch_graph_state)."""
        v = ctypes.c_int()
        _check(lib().fem_batch_graph_state(self._h, ctypes.byref(v)))
        return v.value

    def barrier_selftest(self, timeout_ms=300.0):
        """Status code returned when the persistent kernel's barrier is made
        to wait for an arrival that never comes (FEM_ETIMEOUT expected)."""
        return lib().fem_batch_barrier_selftest(self._h, timeout_ms)


class Mlp:
    """Per-element perceptron n_in -> n_h -> n_h -> n_out (ReLU), FP32 master
    weights; mode 0 = bf16 tensor-core GEMMs, 1 = FP32 (fem_mlp_*)."""

    def __init__(self, n_in, n_h, n_out, params, mode=0, stream=None):
        self.n_in, self.n_h, self.n_out, self.mode = n_in, n_h, n_out, mode
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = _VP()
        _check(lib().fem_mlp_create(n_in, n_h, n_out, mode, _ptr(p), _stream_handle(stream),
                                    ctypes.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fem_mlp_destroy(self._h)
            self._h = None

    def save(self, path):
        """Parameters, Adam moments and step count to a file (fem_mlp_save)."""
        _check(lib().fem_mlp_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path, stream=None):
        """A network restored from fem_mlp_save's file (fem_mlp_load)."""
        import struct
        h = _VP()
        _check(lib().fem_mlp_load(os.fsencode(path), _stream_handle(stream), ctypes.byref(h)))
        with open(path, "rb") as f:
            n_in, n_h, n_out, mode = struct.unpack("<4i", f.read(24)[8:24])
        self = cls.__new__(cls)
        self.n_in, self.n_h, self.n_out, self.mode = n_in, n_h, n_out, mode
        self._h = h
        return self

    @property
    def input_dtype(self):
        import torch
        return torch.bfloat16 if self.mode == 0 else torch.float32

    def params(self):
        n = ctypes.c_int64()
        _check(lib().fem_mlp_params(self._h, None, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.float32)
        _check(lib().fem_mlp_params(self._h, _ptr(out), ctypes.byref(n)))
        return out

    def _xt(self, X, T=None):
        """Pointers of X [S][n_in] (input dtype) and T [S][n_out] (fp32)."""
        import torch
        S = X.shape[0]
        px = _vec(X, self.input_dtype, S * self.n_in, "X")
        pt = None if T is None else _vec(T, torch.float32, S * self.n_out, "T")
        return S, px, pt

    def forward(self, X):
        import torch
        S, px, _ = self._xt(X)
        Y = torch.empty(S, self.n_out, dtype=torch.float32, device=X.device)
        _check(lib().fem_mlp_forward(self._h, px, S, _ptr(Y)))
        return Y

    def gradient(self, X, T, valid):
        """(loss, FP32 gradient) without updating."""
        g = np.zeros(self.params().size, dtype=np.float32)
        L = ctypes.c_double()
        S, px, pt = self._xt(X, T)
        _check(lib().fem_mlp_train_step(self._h, px, pt, S, valid, 0.0, _ptr(g), ctypes.byref(L)))
        return L.value, g

    def step(self, X, T, valid, lr):
        L = ctypes.c_double()
        S, px, pt = self._xt(X, T)
        _check(lib().fem_mlp_train_step(self._h, px, pt, S, valid, lr, None, ctypes.byref(L)))
        return L.value

    def train_plateau(self, X, T, valid, max_epochs=60, chunk=4, rel_tol=0.01, batch=4096,
                      lr=1e-3, seed=0):
        """Train until the loss stops falling (fem_mlp_train_plateau); returns
        the per-epoch mean losses of the epochs run."""
        S, px, pt = self._xt(X, T)
        losses = np.zeros(max_epochs)
        ran = ctypes.c_int()
        _check(lib().fem_mlp_train_plateau(self._h, px, pt, S, valid, int(max_epochs), int(chunk),
                                           float(rel_tol), int(batch), float(lr), int(seed),
                                           _ptr(losses), ctypes.byref(ran)))
        return losses[:ran.value]

    def train(self, X, T, valid, epochs, batch=4096, lr=1e-3, seed=0):
        losses = np.zeros(epochs)
        S, px, pt = self._xt(X, T)
        _check(lib().fem_mlp_train(self._h, px, pt, S, valid, epochs, batch, lr, seed, _ptr(losses)))
        return losses


class Precond:
    """Jacobi + learned per-element correction (fem_precond_*); mlp=None
    gives the Jacobi part alone."""

    def __init__(self, op, mlp=None):
        self.op, self.mlp = op, mlp
        h = _VP()
        _check(lib().fem_precond_create(op._h, None if mlp is None else mlp._h, ctypes.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fem_precond_destroy(self._h)
            self._h = None

    def features(self):
        out = np.zeros((self.op.E, 32), dtype=np.float32)
        _check(lib().fem_precond_features(self._h, _ptr(out)))
        return out

    def samples(self, b, x_star, x_k, X, T):
        import torch
        n, E = self.op.n, self.op.E
        if self.mlp is None:
            raise ValueError("samples need a network")
        _check(lib().fem_precond_samples(
            self._h, _vec(b, torch.float64, n, "b"), _vec(x_star, torch.float64, n, "x_star"),
            _vec(x_k, torch.float64, n, "x_k"), _vec(X, self.mlp.input_dtype, E * self.mlp.n_in, "X"),
            _vec(T, torch.float32, E * self.mlp.n_out, "T")))

    def set_gamma(self, gamma):
        _check(lib().fem_precond_set_gamma(self._h, float(gamma)))
        self.gamma = float(gamma)

    def calibrate(self, b, gammas=(1.0, 0.5, 0.25, 0.1, 0.0), probe_iters=64):
        """Pick the learned-term weight among `gammas` (fem_precond_calibrate)."""
        import torch
        g = np.ascontiguousarray(gammas, dtype=np.float64)
        x = torch.zeros_like(b)
        best = ctypes.c_double()
        _check(lib().fem_precond_calibrate(self._h, _vec(b, torch.float64, self.op.n, "b"),
                                           _vec(x, torch.float64, self.op.n, "x"), _ptr(g), g.size,
                                           int(probe_iters), ctypes.byref(best)))
        return best.value

    def apply(self, r):
        import torch
        z = torch.empty_like(r)
        _check(lib().fem_precond_apply(self._h, _vec(r, torch.float32, self.op.n, "r"),
                                       _vec(z, torch.float32, self.op.n, "z")))
        return z

    def fcg(self, b, x, rtol=1e-10, inner_rtol=0.1, maxit=100000, max_outer=100):
        o = _CgOpts(PC_LEARNED, int(maxit), float(rtol), 1, float(inner_rtol), int(max_outer))
        st = _CgStats()
        import torch
        rc = lib().fem_fcg_solve(self._h, _vec(b, torch.float64, self.op.n, "b"),
                                 _vec(x, torch.float64, self.op.n, "x"), ctypes.byref(o), ctypes.byref(st))
        if rc not in (0, 5):
            _check(rc)
        return _stats(st)


class Pmg:
    """p-multigrid hierarchy over operators of decreasing order on the same
    elements (include/fem.h, fem_pmg_*): Chebyshev-Jacobi smoothing,
    interpolation transfers, Jacobi-PCG on the coarsest level; flexible CG
    around one V-cycle per iteration.  `levels` finest first; the operators
    must outlive this object."""

    def __init__(self, levels, cheb_degree=4, cheb_lo=0.1, cheb_hi=1.1, power_its=20,
                 coarse_its=30, prec=F64):
        self.levels = list(levels)
        arr = (_VP * len(self.levels))(*[o._h for o in self.levels])
        o = _PmgOpts(int(cheb_degree), float(cheb_lo), float(cheb_hi), int(power_its),
                     int(coarse_its), int(prec))
        h = _VP()
        _check(lib().fem_pmg_create(arr, len(self.levels), ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_pc", None) and _lib is not None:
            _lib.fem_precond_destroy(self._pc)
            self._pc = None
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fem_pmg_destroy(self._h)
            self._h = None

    def lmax(self, level):
        v = ctypes.c_double()
        _check(lib().fem_pmg_get_lmax(self._h, int(level), ctypes.byref(v)))
        return v.value

    def set_lmax(self, level, value):
        _check(lib().fem_pmg_set_lmax(self._h, int(level), float(value)))

    def prolong(self, level, xc):
        import torch
        xf = torch.empty(self.levels[level].n, dtype=torch.float64, device=xc.device)
        _check(lib().fem_pmg_prolong(self._h, int(level),
                                     _vec(xc, torch.float64, self.levels[level + 1].n, "xc"),
                                     _vec(xf, torch.float64, self.levels[level].n, "xf")))
        return xf

    def restrict(self, level, rf):
        import torch
        rc = torch.empty(self.levels[level + 1].n, dtype=torch.float64, device=rf.device)
        _check(lib().fem_pmg_restrict(self._h, int(level),
                                      _vec(rf, torch.float64, self.levels[level].n, "rf"),
                                      _vec(rc, torch.float64, self.levels[level + 1].n, "rc")))
        return rc

    def vcycle(self, r):
        import torch
        z = torch.empty_like(r)
        _check(lib().fem_pmg_vcycle(self._h, _vec(r, torch.float64, self.levels[0].n, "r"),
                                    _vec(z, torch.float64, self.levels[0].n, "z")))
        return z

    def solve(self, b, x, rtol=1e-10, maxit=1000):
        o = _CgOpts(0, int(maxit), float(rtol), 1, 0.0, 0)
        st = _CgStats()
        import torch
        n = self.levels[0].n
        rc = lib().fem_pmg_solve(self._h, _vec(b, torch.float64, n, "b"), _vec(x, torch.float64, n, "x"),
                                 ctypes.byref(o), ctypes.byref(st))
        if rc not in (0, 5):
            _check(rc)
        return _stats(st)

    def _precond(self):
        if getattr(self, "_pc", None) is None:
            h = _VP()
            _check(lib().fem_precond_create_pmg(self._h, ctypes.byref(h)))
            self._pc = h
        return self._pc

    def vcycle_f32(self, r):
        """z = V(r) through the FP32 preconditioner object (FP32 [n] in/out)."""
        import torch
        n = self.levels[0].n
        z = torch.empty_like(r)
        _check(lib().fem_precond_apply(self._precond(), _vec(r, torch.float32, n, "r"),
                                       _vec(z, torch.float32, n, "z")))
        return z

    def solve_refined(self, b, x, rtol=1e-10, inner_rtol=1e-4, maxit=1000, max_outer=50):
        """Flexible CG in FP32 around the FP32 V-cycle, inside FP64 iterative
        refinement (fem_precond_create_pmg + fem_fcg_solve); needs prec=F32."""
        import torch
        n = self.levels[0].n
        o = _CgOpts(PC_LEARNED, int(maxit), float(rtol), 1, float(inner_rtol), int(max_outer))
        st = _CgStats()
        rc = lib().fem_fcg_solve(self._precond(), _vec(b, torch.float64, n, "b"),
                                 _vec(x, torch.float64, n, "x"), ctypes.byref(o), ctypes.byref(st))
        if rc not in (0, 5):
            _check(rc)
        return _stats(st)


def pcg_dist(op, owned, b, x, y, sum_interfaces, allreduce, precond=PC_JACOBI, rtol=1e-10,
             maxit=10000, zero_guess=True):
    """One rank's element-partitioned PCG (fem_pcg_dist); sum_interfaces and
    allreduce are _CommSum / _CommReduce callbacks (paper_2109_04996_b300.dist
    builds them from torch.distributed)."""
    import torch
    comm = _Comm(None, sum_interfaces, allreduce)
    o = _CgOpts(precond, int(maxit), float(rtol), 0, 0.0, 0, 1 if zero_guess else 0)
    st = _CgStats()
    rc = lib().fem_pcg_dist(op._h, _vec(owned, torch.uint8, op.N, "owned"),
                            _vec(b, torch.float64, op.n, "b"), _vec(x, torch.float64, op.n, "x"),
                            _vec(y, torch.float64, op.n, "y"), ctypes.byref(o), ctypes.byref(comm),
                            ctypes.byref(st))
    if rc not in (0, 5):
        _check(rc)
    return _stats(st)

"""The allocation-free CG entry point (fem_cg_solve_noalloc).

Callers that cannot allocate device memory while solving (a device-memory
budget fixed at start-up, a real-time loop that cannot afford cudaMalloc's
implicit device-wide synchronization) use this variant of fem_cg_solve whose
workspace is a fixed device array inside the library.  This file checks,
through the C ABI, that two calls in a row give the results of the existing
fem_cg_solve, and that a system larger than the fixed workspace is refused.
It is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest
import torch

import fem_inputs
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

pytestmark = pytest.mark.gpu

MAX_N = 131072  # FEM_NOALLOC_MAX_N in include/fem.h


@pytest.fixture(scope="module")
def L():
    fembuild.build()
    assert torch.cuda.is_available()
    L = fem.lib()
    L.fem_cg_solve_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(fem._CgOpts), ctypes.POINTER(fem._CgStats)]
    L.fem_cg_solve_noalloc.restype = ctypes.c_int
    return L


def _solve(L, fn, op, b, x, precond, maxit, rtol, use_graph=1, zero_guess=0):
    o = fem._CgOpts(precond, maxit, rtol, use_graph, 0.0, 0, zero_guess)
    st = fem._CgStats()
    rc = getattr(L, fn)(op._h, b.data_ptr(), x.data_ptr(), ctypes.byref(o), ctypes.byref(st))
    return rc, st


@pytest.mark.parametrize("name,p,n,precond,rtol,maxit", [
    ("BP3", 3, 4, fem.PC_JACOBI, 1e-10, 10000),
    ("BP6", 2, 3, fem.PC_JACOBI, 1e-10, 10000),
    ("BP1", 2, 8, fem.PC_NONE, 0.0, 100),
])
def test_noalloc_matches_cg_solve_twice_in_a_row(L, name, p, n, precond, rtol, maxit):
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=21)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, name)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=22,
                                                ncomp=op.ncomp)).cuda()
    xr = torch.zeros_like(b)
    rc, st_ref = _solve(L, "fem_cg_solve", op, b, xr, precond, maxit, rtol)
    assert rc == 0, L.fem_last_error()
    for _ in range(2):
        x = torch.zeros_like(b)
        rc, st = _solve(L, "fem_cg_solve_noalloc", op, b, x, precond, maxit, rtol)
        assert rc == 0, L.fem_last_error()
        assert st.iterations == st_ref.iterations
        err = torch.linalg.norm(x - xr).item() / torch.linalg.norm(xr).item()
        assert err <= 1e-12
        assert abs(st.rnorm - st_ref.rnorm) <= 1e-12 * st_ref.bnorm
        if rtol == 0.0:
            assert st.iterations == maxit


@pytest.mark.parametrize("zero_guess", [0, 1])
def test_noalloc_initial_guess_as_cg_solve(L, zero_guess):
    """zero_guess = 1 ignores x on entry (NaN here); zero_guess = 0 starts from
    it (a random x0).  Both against fem_cg_solve with the same options, on
    iterations and solution, and the zero-guess solution against the oracle's
    Jacobi-PCG."""
    import oracle
    m = fem_inputs.box_mesh(4, 3, perturb=0.1, seed=23, shuffle_seed=5)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, "BP3")
    bn = fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=24)
    b = torch.from_numpy(bn).cuda()
    if zero_guess:
        x0 = torch.full_like(b, float("nan"))
    else:
        x0 = torch.from_numpy(np.random.default_rng(25).uniform(-1, 1, m["N"])).cuda()
        x0[torch.from_numpy(m["dirichlet"]).cuda().bool()] = 0.0
    xr = x0.clone()
    rc, st_ref = _solve(L, "fem_cg_solve", op, b, xr, fem.PC_JACOBI, 10000, 1e-10,
                        zero_guess=zero_guess)
    assert rc == 0, L.fem_last_error()
    for _ in range(2):
        x = x0.clone()
        rc, st = _solve(L, "fem_cg_solve_noalloc", op, b, x, fem.PC_JACOBI, 10000, 1e-10,
                        zero_guess=zero_guess)
        assert rc == 0, L.fem_last_error()
        assert st.iterations == st_ref.iterations
        assert torch.isfinite(x).all()
        err = torch.linalg.norm(x - xr).item() / torch.linalg.norm(xr).item()
        assert err <= 1e-12
    if zero_guess:
        orc = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, 5)
        xo, it_o, _ = oracle.pcg(orc, bn, m["dirichlet"], rtol=1e-10)
        assert abs(st.iterations - it_o) <= 2
        xc = x.cpu().numpy()
        assert np.linalg.norm(xc - xo) <= 1e-8 * np.linalg.norm(xo)


def test_noalloc_refuses_systems_beyond_its_workspace(L):
    m = fem_inputs.box_mesh(17, 3, perturb=0.0)     # N = 52^3 = 140608 > MAX_N
    assert m["N"] > MAX_N
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, "BP3")
    b = torch.zeros(m["N"], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    rc, _ = _solve(L, "fem_cg_solve_noalloc", op, b, x, fem.PC_JACOBI, 10, 1e-8)
    assert rc == 1
    assert b"exceeds the fixed workspace" in L.fem_last_error()

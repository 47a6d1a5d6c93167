"""CPU-side checks of the C ABI: the library loads, exports every entry point
declared in include/fem.h, its host-side tables agree with the oracle's, and
argument errors come back as status codes (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import fem_inputs
import oracle
import paper_2109_04996_b300 as fem
from paper_2109_04996_b300 import build as fembuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    fembuild.build()
    return fem.lib()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fem_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("quad", [fem.GAUSS, fem.LOBATTO])
@pytest.mark.parametrize("p", range(1, 9))
def test_basis_tables_match_oracle(L, p, quad):
    for q in ([p + 1, p + 2] if quad == fem.GAUSS else [p + 1]):
        t = fem.basis_tables(p, q, quad)
        z, _ = oracle.gauss_lobatto(p + 1)
        r, w = oracle.gauss_legendre(q) if quad == fem.GAUSS else oracle.gauss_lobatto(q)
        np.testing.assert_allclose(t["nodes"], z, atol=1e-15)
        np.testing.assert_allclose(t["qpts"], r, atol=1e-15)
        np.testing.assert_allclose(t["qwts"], w, atol=1e-15)
        v, d = oracle.lagrange_1d(p, r)
        np.testing.assert_allclose(t["interp"], v, atol=1e-14)
        np.testing.assert_allclose(t["grad"], d, atol=1e-12)


def test_basis_tables_reject_bad_orders(L):
    for p, q, quad in [(0, 2, 0), (9, 11, 0), (3, 7, 0), (3, 5, 1), (3, 4, 7)]:
        with pytest.raises(fem.FemError) as ei:
            fem.basis_tables(p, q, quad)
        assert ei.value.code == 1 and "unsupported" in str(ei.value)


@pytest.mark.parametrize("p", [1, 3, 8])
def test_node_coordinates_match_oracle(L, p):
    m = fem_inputs.box_mesh(3, p, perturb=0.1, seed=9, shuffle_seed=4)
    np.testing.assert_allclose(fem.nodes_from_vertices(m), oracle.nodes_from_vertices(m),
                               rtol=0, atol=2e-16 * 4)


def test_mesh_create_rejects_bad_input_without_a_gpu(L):
    m = fem_inputs.box_mesh(2, 2)
    en = np.ascontiguousarray(m["elem_nodes"]).copy()
    xyz = np.zeros((m["N"], 3))
    h = ctypes.c_void_p()
    rc = L.fem_mesh_create(0, m["N"], m["E"], en.ctypes.data, xyz.ctypes.data, None, None,
                           ctypes.byref(h))
    assert rc == 1 and b"p=0" in L.fem_last_error()
    en[3, 5] = m["N"]
    rc = L.fem_mesh_create(2, m["N"], m["E"], en.ctypes.data, xyz.ctypes.data, None, None,
                           ctypes.byref(h))
    assert rc == 1 and b"out of" in L.fem_last_error()
    rc = L.fem_op_create(None, 1, 0, 4, 1, 0, None, 0, 1.0, ctypes.byref(h))
    assert rc == 1


def test_mesh_box_rejects_bad_arguments_without_a_gpu(L):
    h = ctypes.c_void_p()
    f = L.fem_mesh_box
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                  ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert f(0, 2, 2, 2, 0.1, 0, None, ctypes.byref(h)) == 1
    assert f(9, 2, 2, 2, 0.1, 0, None, ctypes.byref(h)) == 1
    assert f(2, 0, 2, 2, 0.1, 0, None, ctypes.byref(h)) == 1
    assert f(2, 2, 2, 2, 0.5, 0, None, ctypes.byref(h)) == 1
    assert f(2, 2, 2, 2, -0.1, 0, None, ctypes.byref(h)) == 1
    assert b"perturb" in L.fem_last_error()
    assert f(8, 2000, 2000, 2000, 0.0, 0, None, ctypes.byref(h)) == 1
    assert b"int32" in L.fem_last_error()
    assert f(2, 2, 2, 2, 0.1, 0, None, None) == 1


def test_pmg_create_rejects_bad_hierarchies_without_a_gpu(L):
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.fem_pmg_create(arr, 0, None, ctypes.byref(h)) == 1
    assert L.fem_pmg_create(arr, 9, None, ctypes.byref(h)) == 1
    assert L.fem_pmg_create(arr, 2, None, ctypes.byref(h)) == 1
    assert b"level 0" in L.fem_last_error()
    assert L.fem_pmg_vcycle(None, None, None) == 1
    assert L.fem_pmg_solve(None, None, None, None, None) == 1


def test_binding_validates_buffers_before_the_library_sees_them():
    import torch
    with pytest.raises(ValueError, match="CUDA tensor"):
        fem._vec(torch.zeros(8, dtype=torch.float64), torch.float64, 8)
    with pytest.raises(ValueError, match="CUDA tensor"):
        fem._vec(np.zeros(8), torch.float64, 8)
    with pytest.raises(ValueError, match="contiguous"):
        fem._ptr(np.zeros((4, 4))[:, 1])
    m = fem_inputs.box_mesh(2, 2)
    bad = dict(m, elem_nodes=m["elem_nodes"][:-1])
    with pytest.raises(ValueError, match="elem_nodes"):
        fem.Mesh(bad)
    bad = dict(m, dirichlet=m["dirichlet"][:-3])
    with pytest.raises(ValueError, match="dirichlet"):
        fem.Mesh(bad)
    bad = dict(m, elem_verts=m["elem_verts"][:, :7])
    with pytest.raises(ValueError, match="elem_verts"):
        fem.Mesh(bad)

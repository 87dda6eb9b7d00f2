"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and
its task scheduler (run by the host reference executor) reproduces the
recursive H-LU.  No GPU is used."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2211_11303_gb300 import hlu
    return hlu.lib()


def _declared():
    names = []
    for h in ("hlu.h", "hlu_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"^\s*typedef [^;{]*\(\*\w+\)\([^;]*\);", "", src, flags=re.M)  # function-pointer types
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "sizeof", "defined"):
                names.append(name)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_2211_11303_gb300 import hlu
    declared = _declared()
    assert "hlu_build" in declared and "gmres_solve" in declared
    for name in declared:
        assert hasattr(lib, name), name
        assert name in hlu.SIGNATURES, name


def test_status_strings(lib):
    assert lib.hlu_status_string(0) == b"HLU_OK"
    assert lib.hlu_status_string(5) == b"HLU_ERR_TIMEOUT"


def test_build_rejects_bad_arguments(lib):
    from paper_2211_11303_gb300 import hlu
    h = ctypes.c_void_p()
    m = hlu.lattice_mesh(0)  # neither a lattice nor a general mesh
    assert lib.hlu_build(ctypes.byref(m), 1.0, 32, 2.0, 1e-4, 32, None, ctypes.byref(h)) == 1
    m = hlu.lattice_mesh(4)
    assert lib.hlu_build(ctypes.byref(m), 1.0, 32, 1.5, 1e-4, 32, None, ctypes.byref(h)) == 1  # eta^2 = 2.25
    assert lib.hlu_build(None, 1.0, 32, 2.0, 1e-4, 32, None, ctypes.byref(h)) == 1


def _host_solve(lib, n, kappa, eps, leaf, seed, nrhs=2, tile=0, precision=0):
    from oracle import fem, mesh, trees
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    perm, cl, bl = trees.build_trees(m, leaf, 2.0)
    p, C, B = trees.export_arrays(perm, cl, bl)
    N = A.shape[0]
    rng = np.random.default_rng(1)
    b = np.asfortranarray(rng.standard_normal((N, nrhs)))
    x = np.zeros((N, nrhs), order="F")
    info = np.zeros(10, dtype=np.int64)
    rp = A.indptr.astype(np.int64)
    ci = A.indices.astype(np.int32)
    va = A.data.astype(np.float64)
    st = lib.hlu_debug_host_factor_solve(len(C), C.ctypes.data, len(B), B.ctypes.data, p.ctypes.data,
                                         rp.ctypes.data, ci.ctypes.data, va.ctypes.data, eps, 32, tile, precision, seed,
                                         nrhs, b.ctypes.data, x.ctypes.data, info.ctypes.data)
    assert st == 0
    return A, perm, cl, bl, b, x, info


def test_dag_any_topological_order_is_bit_identical(lib):
    _, _, _, _, _, x0, info = _host_solve(lib, 4, 3.0, 1e-4, 16, 0)
    for seed in (1, 2, 3):
        _, _, _, _, _, x1, _ = _host_solve(lib, 4, 3.0, 1e-4, 16, seed)
        assert np.array_equal(x0, x1)
    assert info[0] > 0 and info[1] > 0


@pytest.mark.parametrize("n,kappa,leaf", [(4, 1.0, 16), (5, 4.0, 16)])
def test_scheduled_hlu_matches_recursive_oracle(lib, n, kappa, leaf):
    from oracle import hmatrix
    for eps in (1e-12, 1e-4):
        A, perm, cl, bl, b, x, info = _host_solve(lib, n, kappa, eps, leaf, 0)
        P = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
        xo = P.apply(b)
        xs = np.linalg.solve(A.toarray(), b)
        e_lib = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        e_or = np.linalg.norm(xo - xs) / np.linalg.norm(xs)
        if eps < 1e-10:
            assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)
        else:
            assert e_lib <= 2.0 * e_or + 1e-12, (e_lib, e_or)


@pytest.mark.parametrize("n,kappa,leaf,tile", [(4, 3.0, 8, 16), (5, 5.0, 8, 32), (5, 5.0, 16, 64)])
def test_tiled_factor_tree_quality(lib, n, kappa, leaf, tile):
    """Dense tiles above the leaf level keep exactness inside the tile, so the
    factor is at least as accurate as the leaf-level recursive H-LU."""
    from oracle import hmatrix
    for eps in (1e-12, 1e-3):
        A, perm, cl, bl, b, x, info = _host_solve(lib, n, kappa, eps, leaf, 0, tile=tile)
        xs = np.linalg.solve(A.toarray(), b)
        e_lib = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        P = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
        e_or = np.linalg.norm(P.apply(b) - xs) / np.linalg.norm(xs)
        assert e_lib <= 2.0 * e_or + 1e-11, (eps, e_lib, e_or)
    _, _, _, _, _, x2, _ = _host_solve(lib, n, kappa, 1e-3, leaf, 9, tile=tile)
    _, _, _, _, _, x3, _ = _host_solve(lib, n, kappa, 1e-3, leaf, 0, tile=tile)
    assert np.array_equal(x2, x3)


def test_allocator_and_memory_limit_arguments(lib):
    """hlu_set_allocator takes both callbacks or neither; the memory limit is
    a non-negative byte count (no device needed)."""
    from paper_2211_11303_gb300 import hlu
    cb = hlu._ALLOC_FN(lambda n, ctx: None)
    assert lib.hlu_set_allocator(ctypes.cast(cb, ctypes.c_void_p), None, None) == 1
    assert lib.hlu_set_device_memory_limit(-1) == 1
    assert lib.hlu_set_device_memory_limit(0) == 0
    assert lib.hlu_device_bytes_in_use() >= 0


def test_kuhn_cube_mesh_export_matches_the_input_recipe(lib):
    """hlu_mesh_kuhn_cube (host arrays, no device) lists the same vertices and
    tetrahedra, in the same order, as the seeded mesh recipe of the tests and
    the oracle's Kuhn cube."""
    import synth
    from oracle import mesh
    from paper_2211_11303_gb300 import hlu
    for n in (1, 2, 5):
        xyz, tets = hlu.hlu_mesh_kuhn_cube(n)
        c, t = synth.perturbed_kuhn_mesh(n, 0.0, 1)
        assert np.array_equal(tets, t) and np.array_equal(xyz, c)
        lat, ot = mesh.kuhn_cube(n)
        assert np.array_equal(tets, ot) and np.array_equal(xyz, lat / float(n))


def test_general_mesh_arguments_are_checked(lib):
    """Invalid general meshes are refused before any device work."""
    from paper_2211_11303_gb300 import hlu
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=np.float64)
    good = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    h = ctypes.c_void_p()

    def build(x, t):
        x = np.ascontiguousarray(x, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.int32)
        m = hlu.hlu_mesh(x.shape[0], t.shape[0], x.ctypes.data, t.ctypes.data, 0)
        return lib.hlu_build(ctypes.byref(m), 1.0, 32, 2.0, 1e-4, 0, None, ctypes.byref(h))

    assert build(xyz, np.array([[0, 1, 2, 5]])) == 1       # vertex id out of range
    assert build(xyz, np.array([[0, 1, 1, 3]])) == 1       # repeated vertex
    bad = xyz.copy()
    bad[4, 2] = np.nan
    assert build(bad, good) == 1                           # non-finite coordinate
    assert build(xyz[:3], np.array([[0, 1, 2, 0]])) == 1   # fewer than 4 vertices
    # a material coefficient must be finite and positive on every tetrahedron
    for bad_beta in ([1.0, 0.0], [1.0, -2.0], [np.nan, 1.0]):
        bb = np.ascontiguousarray(bad_beta, dtype=np.float64)
        x = np.ascontiguousarray(xyz)
        m = hlu.hlu_mesh(x.shape[0], good.shape[0], x.ctypes.data, good.ctypes.data, 0, bb.ctypes.data)
        assert lib.hlu_build(ctypes.byref(m), 1.0, 32, 2.0, 1e-4, 0, None, ctypes.byref(h)) == 1
    bl = np.full(6 * 2 ** 3, 1.0)
    bl[5] = np.inf
    m = hlu.lattice_mesh(2, bl)
    assert lib.hlu_build(ctypes.byref(m), 1.0, 32, 2.0, 1e-4, 0, None, ctypes.byref(h)) == 1


def test_example3_magnet_matches_oracle(lib):
    """The Example 3 driver's magnet coefficient (from the library's Kuhn
    cube export) equals the oracle's (from its own mesh), tetrahedron by
    tetrahedron, at a size where the box faces are lattice planes and one
    where they are not."""
    from oracle import fem, mesh
    from paper_2211_11303_gb300 import example3
    for n in (8, 6):
        b = example3.magnet_beta(n)
        bo = fem.magnet_beta(mesh.interior_edges(n), 10.0)
        assert np.array_equal(b, bo)

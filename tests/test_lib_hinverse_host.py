"""The Schulz inverse's task DAGs (the schedules hlu_hinverse runs on the
GPU) executed by the library's host reference executor in FP64, against the
oracle's Schulz iteration and the exact inverse.  No GPU."""
import ctypes

import numpy as np
import pytest

from oracle import fem, hinverse, mesh, trees


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2211_11303_gb300 import hlu
    return hlu.lib()


def _host_inverse(lib, A, perm, cl, bl, eps, iters, Z, tile=0):
    p, C, B = trees.export_arrays(perm, cl, bl)
    C = np.ascontiguousarray(C, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.int32)
    p = np.ascontiguousarray(p, dtype=np.int32)
    rp, ci, va = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)
    Ad = A.toarray()
    alpha = 1.0 / (np.abs(Ad).sum(0).max() * np.abs(Ad).sum(1).max())
    Zf = np.asfortranarray(Z)
    X = np.zeros_like(Zf)
    info = (ctypes.c_int64 * 5)()
    rc = lib.hlu_debug_host_hinverse(len(C), C.ctypes.data, len(B), B.ctypes.data, p.ctypes.data, rp.ctypes.data,
                                     ci.ctypes.data, va.ctypes.data, eps, 0, tile, alpha, iters, Z.shape[1],
                                     Zf.ctypes.data, X.ctypes.data, info)
    assert rc == 0
    return X, list(info)


@pytest.mark.parametrize("tile", [0, 64])
def test_host_schulz_dags_reach_the_exact_inverse(lib, tile):
    n, kappa, leaf = 3, 1.5, 8
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    perm, cl, bl = trees.build_trees(m, leaf, 2.0)
    Z = np.random.default_rng(1).standard_normal((A.shape[0], 3))
    X, info = _host_inverse(lib, A, perm, cl, bl, 1e-14, 32, Z, tile)
    Xs = np.linalg.solve(A.toarray(), Z)
    assert np.linalg.norm(X - Xs) <= 1e-9 * np.linalg.norm(Xs)
    assert info[3] == 0  # no rank-capacity hit



@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_host_schulz_dags_within_2x_of_oracle(lib, eps):
    """After the same number of steps, ||z - A X z|| / ||z|| of the DAGs'
    iterate (formatted H-arithmetic) is within 2x of the oracle's (exact
    products projected onto the H-format)."""
    n, kappa, leaf = 4, 3.0, 16
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    perm, cl, bl = trees.build_trees(m, leaf, 2.0)
    N = A.shape[0]
    Z = np.random.default_rng(2).standard_normal((N, 4))
    B, info_or = hinverse.schulz_inverse(A, perm, cl, bl, eps=eps, tol=1e-14, maxit=40)
    X, info = _host_inverse(lib, A, perm, cl, bl, eps, info_or["iters"], Z)
    err = lambda Y: max(np.linalg.norm((Z - A @ Y)[:, i]) / np.linalg.norm(Z[:, i]) for i in range(4))
    e_or, e_dag = err(B @ Z), err(X)
    assert e_dag <= 2.0 * e_or, (e_dag, e_or)

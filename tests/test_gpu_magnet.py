"""GPU parity with a material coefficient (Sec. 2: the operator
curl(beta^-1 curl E) - kappa E; Sec. 4, Example 3: a magnet with beta = 10 in
air, kappa = 10, J_S = [10, 10, 10]^T, Algorithm 1 to TOL 1e-8).

The magnet stand-in is the centred 0.5 x 0.5 x 0.75 box in the Kuhn cube
(oracle.fem.magnet_beta); the paper's own Netgen mesh is not available.  The
assembled matrix is held to the oracle's element by element, the
preconditioned Richardson iteration (Algorithm 1 steps III-IV) to the direct
solve of the oracle's matrix, and its iteration count to the oracle's own
Richardson iteration with its own H-LU.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem, hmatrix, krylov, mesh, trees

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA = math.sqrt(10.0)  # the paper's kappa = 10 is kappa^2 here
J_S = (10.0, 10.0, 10.0)


@pytest.fixture(scope="module")
def hlu():
    import __graft_entry__ as g
    g.build()
    from paper_2211_11303_gb300 import hlu as H
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    H.hlu_set_wait_limit_ms(20000)
    return H


@pytest.mark.parametrize("n", [4, 8])
def test_magnet_assembly_matches_oracle(hlu, n):
    m = mesh.interior_edges(n)
    beta = fem.magnet_beta(m, 10.0)
    A = fem.assemble(m, KAPPA, beta=beta).tocsr()
    h = hlu.hlu_build(n, KAPPA, 32, 2.0, 1e-4, beta=beta)
    try:
        rp, ci, va = hlu.hlu_export_csr(h)
        assert np.array_equal(rp, A.indptr.astype(np.int64))
        assert np.array_equal(ci, A.indices.astype(np.int32))
        assert np.abs(va - A.data).max() <= 1e-13 * np.abs(A.data).max()
    finally:
        hlu.hlu_destroy(h)


def test_magnet_on_a_general_mesh_matches_oracle(hlu):
    coords, tets = synth.perturbed_kuhn_mesh(6, 0.15, 9)
    m = mesh.general_mesh(coords, tets)
    beta = fem.magnet_beta(m, 10.0)
    A = fem.assemble(m, KAPPA, beta=beta).tocsr()
    h = hlu.hlu_build_mesh(coords, tets, KAPPA, 16, 2.0, 1e-4, beta=beta)
    try:
        rp, ci, va = hlu.hlu_export_csr(h)
        assert np.array_equal(rp, A.indptr.astype(np.int64))
        assert np.array_equal(ci, A.indices.astype(np.int32))
        assert np.abs(va - A.data).max() <= 1e-13 * np.abs(A.data).max()
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_example3_richardson(hlu, prec):
    """n = 8 (N = 3,032): Algorithm 1 with the H-LU at eps 1e-4 reaches the
    direct solve to 1e-7, in at most one iteration more than the oracle's
    Richardson iteration with its own H-LU."""
    n, eps = 8, 1e-4
    m = mesh.interior_edges(n)
    beta = fem.magnet_beta(m, 10.0)
    A = fem.assemble(m, KAPPA, beta=beta).tocsr()
    bo = fem.constant_current_rhs(m, J_S)
    h = hlu.hlu_build(n, KAPPA, 32, 2.0, eps, beta=beta)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32)
        N = hlu.hlu_n(h)
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        hlu.hlu_rhs_constant_current(h, J_S, b)
        assert np.abs(b.cpu().numpy() - bo).max() <= 1e-13 * np.abs(bo).max()
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        st = hlu.hlu_richardson(h, b, x, tol=1e-8, maxit=60)
        xs = spla.spsolve(A.tocsc(), bo)
        assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-7 * np.linalg.norm(xs)
        perm, cl, bl = trees.build_trees(m, 32, 2.0)
        xo, info = krylov.richardson(lambda v: A @ v, bo, hmatrix.HLUPreconditioner(A, perm, cl, bl, eps).apply,
                                     tol=1e-8)
        assert st["iterations"] <= info["iters"] + 1, (st["iterations"], info["iters"])
    finally:
        hlu.hlu_destroy(h)

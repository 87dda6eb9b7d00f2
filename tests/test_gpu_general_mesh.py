"""General tetrahedral meshes at the C ABI (hlu_mesh with vertex coordinates
and tetrahedra): a perturbed, non-lattice cube is assembled, clustered and
solved on the GPU and compared with the CPU oracle on the same mesh (Sec.
2.1: a conforming tetrahedral mesh, one DOF per interior edge)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem, hmatrix, mesh, trees

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hlu():
    import __graft_entry__ as g
    g.build()
    from paper_2211_11303_gb300 import hlu as H
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    H.hlu_set_wait_limit_ms(20000)
    return H


@pytest.mark.parametrize("n,amp,seed", [(2, 0.2, 1), (3, 0.2, 2), (5, 0.15, 3), (7, 0.2, 4)])
def test_perturbed_mesh_matches_oracle(hlu, n, amp, seed):
    coords, tets = synth.perturbed_kuhn_mesh(n, amp, seed)
    m = mesh.general_mesh(coords, tets)
    A = fem.assemble(m, 3.0).tocsr()
    perm, cl, bl = trees.build_trees(m, 16, 2.0)
    p, C, B = trees.export_arrays(perm, cl, bl)
    h = hlu.hlu_build_mesh(coords, tets, 3.0, 16, 2.0, 1e-4)
    try:
        assert hlu.hlu_n(h) == A.shape[0] == mesh.n_interior_edges_formula(n)
        rp, ci, va = hlu.hlu_export_csr(h)
        assert np.array_equal(rp, A.indptr.astype(np.int64))
        assert np.array_equal(ci, A.indices.astype(np.int32))
        assert np.abs(va - A.data).max() <= 1e-13 * np.abs(A.data).max()
        gp, gC, gB = hlu.hlu_export_trees(h)
        assert np.array_equal(gp, p) and np.array_equal(gC, C) and np.array_equal(gB, B)
        N = A.shape[0]
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        hlu.hlu_rhs_manufactured(h, b)
        bo = fem.manufactured_rhs(m, 3.0)
        assert np.abs(b.cpu().numpy() - bo).max() <= 1e-13 * np.abs(bo).max()
        hlu.hlu_rhs_constant_current(h, (0.0, 0.0, 1.0), b)
        bo = fem.constant_current_rhs(m, (0.0, 0.0, 1.0))
        assert np.abs(b.cpu().numpy() - bo).max() <= 1e-13 * np.abs(bo).max()
    finally:
        hlu.hlu_destroy(h)


def test_general_path_equals_lattice_path_on_the_cube(hlu):
    """The unperturbed cube through the general path assembles the same
    matrix as the lattice path (the DOF numbering rules agree)."""
    n = 6
    xyz, tets = hlu.hlu_mesh_kuhn_cube(n)
    hg = hlu.hlu_build_mesh(xyz, tets, 2.0, 32, 2.0, 1e-4)
    hl = hlu.hlu_build(n, 2.0, 32, 2.0, 1e-4)
    try:
        a = hlu.hlu_export_csr(hg)
        b = hlu.hlu_export_csr(hl)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.abs(a[2] - b[2]).max() <= 1e-14 * np.abs(b[2]).max()
    finally:
        hlu.hlu_destroy(hg)
        hlu.hlu_destroy(hl)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_perturbed_mesh_solve(hlu, prec):
    """H-LU + FGMRES on a perturbed mesh: operator error within 2x of the
    oracle's recursive H-LU at equal eps, solution within 1e-7 of the direct
    solve."""
    n, kappa, eps = 6, 4.0, 1e-3
    coords, tets = synth.perturbed_kuhn_mesh(n, 0.2, 21)
    m = mesh.general_mesh(coords, tets)
    A = fem.assemble(m, kappa).tocsr()
    N = A.shape[0]
    perm, cl, bl = trees.build_trees(m, 32, 2.0)
    P = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
    Z = np.stack([synth.normal(40 + i, N) for i in range(3)], axis=1)
    AZ = A @ Z
    e_or = max(np.linalg.norm(Z[:, i] - P.apply(AZ[:, i])) / np.linalg.norm(Z[:, i]) for i in range(3))
    h = hlu.hlu_build_mesh(coords, tets, kappa, 32, 2.0, eps)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32)
        b = hlu.colmajor(N, 3)
        b.copy_(torch.from_numpy(np.asfortranarray(AZ)))
        y = hlu.colmajor(N, 3)
        hlu.hlu_solve(h, b, y)
        torch.cuda.synchronize()
        Y = y.cpu().numpy()
        e_gpu = max(np.linalg.norm(Z[:, i] - Y[:, i]) / np.linalg.norm(Z[:, i]) for i in range(3))
        assert e_gpu <= 2.0 * e_or, (e_gpu, e_or)
        B = np.stack([synth.normal(synth.rhs_seed(6, 0, j), N) for j in range(2)], axis=1)
        b2 = hlu.colmajor(N, 2)
        b2.copy_(torch.from_numpy(np.asfortranarray(B)))
        x = hlu.colmajor(N, 2)
        st = hlu.gmres_solve(h, b2, x, restart=50, tol=1e-10, maxit=500)
        torch.cuda.synchronize()
        xs = spla.splu(A.tocsc()).solve(B)
        assert st["converged"] == 1
        xg = x.cpu().numpy()
        for j in range(2):
            assert np.linalg.norm(xg[:, j] - xs[:, j]) <= 1e-7 * np.linalg.norm(xs[:, j])
    finally:
        hlu.hlu_destroy(h)

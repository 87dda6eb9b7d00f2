"""Pins of the oracle's truncation, leaf LU and H-LU (no GPU)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem as F
from oracle import hmatrix as H
from oracle import mesh as M
from oracle import trees as T


def _problem(n, kappa, leaf=32):
    m = M.interior_edges(n)
    A = F.assemble(m, kappa)
    perm, cl, bl = T.build_trees(m, leaf, 2.0)
    return m, A, perm, cl, bl


def test_truncate_known_singular_values():
    rng = np.random.default_rng(0)
    m, n = 60, 45
    U, _ = np.linalg.qr(rng.standard_normal((m, 6)))
    V, _ = np.linalg.qr(rng.standard_normal((n, 6)))
    s = np.array([3.0, 1.0, 2e-2, 4e-4, 2e-4, 1e-9])
    Mx = (U * s) @ V.T
    # split the matrix into a redundant stacked factor form
    X = np.hstack([U * s, U[:, :2]])
    Y = np.hstack([V, np.zeros((n, 2))])
    for eps, r in [(1e-1, 2), (5e-3, 3), (1e-4, 4), (5e-5, 5), (1e-12, 6)]:
        Xt, Yt = H.truncate(X, Y, eps)
        assert Xt.shape[1] == r
        err = np.linalg.norm(Mx - Xt @ Yt.T, 2)
        assert err <= eps * s[0] * (1 + 1e-9)
        tail = s[r] if r < len(s) else 0.0
        assert abs(err - tail) <= 1e-12 * s[0]


def test_truncate_zero_block():
    X, Y = H.truncate(np.zeros((5, 3)), np.ones((4, 3)), 1e-4)
    assert X.shape == (5, 0) and Y.shape == (4, 0)


def test_getrf_matches_partial_pivoting():
    rng = np.random.default_rng(3)
    for n in (1, 5, 32):
        A = rng.standard_normal((n, n))
        LU, p = H.getrf(A)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        assert np.allclose(L @ U, A[p], atol=1e-12)
        P, L2, U2 = sla.lu(A)  # A = P L U, LAPACK partial pivoting
        assert np.allclose(L, L2, atol=1e-12) and np.allclose(U, U2, atol=1e-12)
    with pytest.raises(H.ZeroPivot):
        H.getrf(np.zeros((3, 3)))


def test_fill_is_exact():
    m, A, perm, cl, bl = _problem(4, 2.0, leaf=16)
    Ap = A[perm][:, perm].tocsr()
    Hm = H.HMatrix(cl, bl, 1e-4)
    Hm.fill(Ap)
    assert np.array_equal(Hm.to_dense(0), Ap.toarray())


@pytest.mark.parametrize("n,kappa,leaf", [(4, 1.0, 16), (4, 5.0, 32), (6, 8.0, 32)])
def test_hlu_tight_eps_is_dense_solve(n, kappa, leaf):
    m, A, perm, cl, bl = _problem(n, kappa, leaf)
    P = H.HLUPreconditioner(A, perm, cl, bl, 1e-14)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(A.shape[0])
    x = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(P.apply(b) - x) <= 1e-9 * np.linalg.norm(x)


def test_hlu_error_falls_with_eps():
    m, A, perm, cl, bl = _problem(6, 4.0)
    Ad = A.toarray()
    N = Ad.shape[0]
    errs = []
    for eps in (1e-1, 1e-2, 1e-4, 1e-6):
        P = H.HLUPreconditioner(A, perm, cl, bl, eps)
        E = np.eye(N) - P.apply(Ad)
        errs.append(np.linalg.norm(E, 2))
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[-1] < 1e-3


def test_hlu_blocks_reproduce_dense_lu_with_leaf_pivots():
    # with eps -> 0 the factors are exact: P A_perm = L U with P block diagonal
    m, A, perm, cl, bl = _problem(4, 3.0, leaf=16)
    Ap = A[perm][:, perm].toarray()
    Hm = H.HMatrix(cl, bl, 1e-15)
    Hm.fill(A[perm][:, perm].tocsr())
    Hm.lu(0)
    F_ = Hm.to_dense(0)
    N = F_.shape[0]
    L = np.tril(F_, -1) + np.eye(N)
    U = np.triu(F_)
    # block-diagonal leaf permutation; off-diagonal L blocks stay unpermuted
    p = np.arange(N)
    for b, piv in Hm.piv.items():
        c = Hm.rows(b)
        p[c["offset"]:c["offset"] + c["size"]] = c["offset"] + piv
    Pm = np.eye(N)[p]
    # L_true = P applied to the strictly-lower part outside the diagonal leaves
    Lt = L.copy()
    for b in Hm.piv:
        c = Hm.rows(b)
        o, s = c["offset"], c["size"]
        Lt[o:o + s, :o] = L[o:o + s, :o][Hm.piv[b]]
    assert np.allclose(Lt @ U, Pm @ Ap, atol=1e-9 * abs(Ap).max())

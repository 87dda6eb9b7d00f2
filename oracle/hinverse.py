"""Inverse of the H-matrix approximation by the Schulz iteration (oracle; test
infrastructure only).

Paper: to use the inverse of the H-matrix approximation A_H of the Galerkin
matrix as a preconditioner, the inverse B_H is obtained by the iterative
method of Schulz (Sec. 3); admissible blocks are kept as truncated SVDs
U_r S_r V_r^T (Sec. 4), and the error of B_H falls as the ranks grow
(Example 2).  The Schulz iteration is X_{k+1} = X_k (2 I - A X_k).

Readings (the paper names the method, not its details):
  * each step is T_k = A_H (.) X_k, X_{k+1} = 2 X_k - X_k (.) T_k, where
    (.) is the formatted product: the exact product projected onto the
    H-format of the block tree (dense leaf blocks kept, each admissible block
    replaced by its SVD truncated to s_i > eps s_1, the truncation rule of the
    H-LU);
  * A_H is A itself (its admissible blocks are exactly low rank, as in A_H of
    the H-LU);
  * X_0 = alpha A^T with alpha = 1 / (||A||_1 ||A||_inf), projected: then
    ||I - A X_0||_2 < 1 and the iteration converges (Hotelling-Bodewig,
    Ben-Israel); the paper does not state its start;
  * stop when ||I - A_H X_k||_2 <= tol, after maxit steps, when the residual
    has reached the floor the truncation leaves (below 1/2 and no longer
    falling by a tenth per step), or when it diverges (above 10 or not
    finite; coarse truncations, e.g. eps = 0.1 on small cubes, do).

Pins (tests/test_oracle_hinverse.py): at eps -> 0 the iterate equals the
exact inverse; the residual of the start is below one and, once below one
half, at least squares per step up to rounding; the final residual falls as
eps shrinks.

Everything is dense and in the cluster tree's permuted DOF order: for the
small meshes the oracle is used on.
"""
import numpy as np

from .trees import ADM, DENSE, SUB


def _leaves(blocks, b=0):
    if blocks[b]["kind"] != SUB:
        yield b
        return
    for s in blocks[b]["sons"]:
        yield from _leaves(blocks, s)


def project(M, clusters, blocks, eps):
    """Best approximation of the dense matrix M (permuted order) in the
    H-format of the block tree; returns (dense matrix, ranks of the admissible
    blocks)."""
    out = np.zeros_like(M)
    ranks = {}
    for b in _leaves(blocks):
        r, c = clusters[blocks[b]["row"]], clusters[blocks[b]["col"]]
        rows = slice(r["offset"], r["offset"] + r["size"])
        cols = slice(c["offset"], c["offset"] + c["size"])
        sub = M[rows, cols]
        if blocks[b]["kind"] == DENSE:
            out[rows, cols] = sub
            continue
        U, s, Vt = np.linalg.svd(sub, full_matrices=False)
        k = int(np.sum(s > eps * s[0])) if s.size and s[0] > 0 else 0
        out[rows, cols] = (U[:, :k] * s[:k]) @ Vt[:k]
        ranks[b] = k
    return out, ranks


def schulz_inverse(A, perm, clusters, blocks, eps, tol=1e-10, maxit=100):
    """B_H ~ A^{-1} in the H-format by the Schulz iteration.  A: sparse or
    dense matrix in the original DOF order.  Returns (B_H dense in the
    original order, info dict: residuals ||I - A X_k||_2 per step, iters,
    ranks of the final iterate)."""
    perm = np.asarray(perm, dtype=np.int64)
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A, dtype=np.float64)
    Ap = Ad[np.ix_(perm, perm)]
    N = Ap.shape[0]
    I = np.eye(N)
    alpha = 1.0 / (np.abs(Ap).sum(axis=0).max() * np.abs(Ap).sum(axis=1).max())
    X, ranks = project(alpha * Ap.T, clusters, blocks, eps)
    res = [np.linalg.norm(I - Ap @ X, 2)]
    it = 0
    while res[-1] > tol and it < maxit:
        T, _ = project(Ap @ X, clusters, blocks, eps)
        Xn, rn = project(2.0 * X - X @ T, clusters, blocks, eps)
        r = np.linalg.norm(I - Ap @ Xn, 2)
        if not np.isfinite(r) or r > 10.0:
            break  # diverged: keep the last iterate
        X, ranks = Xn, rn
        res.append(r)
        it += 1
        if res[-2] < 0.5 and r > 0.9 * res[-2]:
            break  # the truncation floor
    B = np.empty_like(X)
    B[np.ix_(perm, perm)] = X
    return B, {"residuals": res, "iters": it, "ranks": ranks, "alpha": alpha}

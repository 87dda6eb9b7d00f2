"""H-matrix approximation A_H, rank truncation, recursive H-LU and the
H-triangular solves (oracle; test infrastructure only).

Paper: Definition 1 (admissible blocks stored as X Y^T of rank r), Sec. 4
(truncated SVD U_r S_r V_r^T of admissible blocks), Algorithm 1 step I (build
A_H), step II (H-LU: for every block row j the blocks L_jk with k < j, then
L_jj U_jj, then U_jk with k > j, every product summed in H-arithmetic), and the
preconditioner application U^-1 (L^-1 r) of step III.  The printed step II is
the block Crout form of the recursive H-LU in the source it cites (Bebendorf,
Sec. 2.9); this module evaluates it by that recursion:

    LU(A) :  LU(A11);  A12 <- L11^-1 P1 A12;  A21 <- A21 U11^-1;
             A22 <- A22 - A21 A12  (truncated);  LU(A22)

Readings (the paper is silent on these):
  * no global pivoting; a dense diagonal leaf is factored with partial
    pivoting inside the leaf (first index of max |a|; of max |Re a| + |Im a|
    for a complex leaf), P L U = A_leaf, L unit lower, U upper.  Off-diagonal
    L blocks are kept unpermuted and the leaf permutation is applied when the
    solve reaches that leaf, which is the same as P A = L U with P block
    diagonal over the leaf clusters;
  * truncation of X Y^T: QR of X and of Y, SVD of R_x R_y^T = U S V^T, keep the
    singular values s_i > eps s_1 (relative, strict), X <- Q_x U_r S_r,
    Y <- Q_y V_r; a zero block truncates to rank 0;
  * complex blocks (Definition 1's X Y^H) are stored as X Y^T with complex X,
    Y (Y^T = the paper's Y^H, conjugated); every step above then holds with
    transposes, not conjugate transposes, and a complex matrix runs the same
    code in complex arithmetic;
  * A_H is exact: a dense leaf holds the CSR entries, an admissible block holds
    X = the unit columns of its nonzero rows and Y^T = those rows;
  * a product of two subdivided blocks into a low-rank target is formed son by
    son (each son sum truncated), then the four sons are agglomerated into one
    X Y^T and truncated (formatted H-multiplication).

Pins (tests/test_oracle_hmatrix.py): truncation returns the exact rank and an
error <= eps s_1 for matrices with prescribed singular values; A_H equals A
entrywise; eps -> 1e-14 reproduces the dense LU solve; ||I - (LU)_H^-1 A||_2
falls as eps shrinks; the leaf getrf equals scipy's partial-pivoting LU.
Complex (tests/test_oracle_complex.py): the same four on complex input, the
leaf getrf equal to LAPACK's complex LU.
"""
import numpy as np
import scipy.linalg as sla

from .trees import ADM, DENSE, SUB


class ZeroPivot(ArithmeticError):
    pass


def truncate(X, Y, eps):
    """Best rank-r approximation of X Y^T with s_i > eps s_1 (Sec. 4 truncated SVD).
    Complex factors (Definition 1) take the same steps: with R_x R_y^T =
    U S V^H, X Y^T = (Q_x U S)(Q_y conj(V))^T, and conj(V) = (V^H)^T is the
    transpose of the SVD's third factor, as for real input."""
    m, n = X.shape[0], Y.shape[0]
    dt = np.result_type(X, Y, np.float64)
    if X.shape[1] == 0 or m == 0 or n == 0:
        return np.zeros((m, 0), dt), np.zeros((n, 0), dt)
    Qx, Rx = np.linalg.qr(X)
    Qy, Ry = np.linalg.qr(Y)
    U, s, Vt = np.linalg.svd(Rx @ Ry.T)
    if s[0] == 0.0:
        return np.zeros((m, 0), dt), np.zeros((n, 0), dt)
    r = int(np.sum(s > eps * s[0]))
    return Qx @ (U[:, :r] * s[:r]), Qy @ Vt[:r].T


def getrf(A):
    """LU with partial pivoting inside a dense leaf.  Returns (LU packed, p) with
    A[p] = L U (p[i] = original row at position i).  The pivot is the first
    entry of largest |a| in the column; for a complex leaf, of largest
    |Re a| + |Im a|, LAPACK's measure for complex pivots."""
    A = np.array(A, dtype=np.result_type(A, np.float64), copy=True)
    cplx = np.iscomplexobj(A)
    n = A.shape[0]
    p = np.arange(n)
    for k in range(n):
        col = A[k:, k]
        q = k + int(np.argmax(np.abs(col.real) + np.abs(col.imag) if cplx else np.abs(col)))
        if A[q, k] == 0.0:
            raise ZeroPivot(k)
        if q != k:
            A[[k, q]] = A[[q, k]]
            p[[k, q]] = p[[q, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, p


class HMatrix:
    """Block-tree storage over the permuted DOF order."""

    def __init__(self, clusters, blocks, eps):
        self.cl = clusters
        self.bl = blocks
        self.eps = eps
        self.D = {}
        self.X = {}
        self.Y = {}
        self.piv = {}
        self.dtype = np.dtype(np.float64)  # complex128 for a complex matrix

    # ---- shape helpers -------------------------------------------------
    def rows(self, b):
        return self.cl[self.bl[b]["row"]]

    def cols(self, b):
        return self.cl[self.bl[b]["col"]]

    def kind(self, b):
        return self.bl[b]["kind"]

    def son(self, b, i, j):
        return self.bl[b]["sons"][2 * i + j]

    def split_rows(self, b):
        """Relative split point of the block's row cluster."""
        c = self.rows(b)
        s0 = self.cl[c["sons"][0]]
        return s0["size"]

    def split_cols(self, b):
        c = self.cols(b)
        return self.cl[c["sons"][0]]["size"]

    # ---- A_H (Alg. 1 step I) --------------------------------------------
    def fill(self, Ap):
        """Ap: CSR matrix already permuted to cluster order."""
        self.dtype = np.result_type(Ap.dtype, np.float64)
        for b, blk in enumerate(self.bl):
            if blk["kind"] == SUB:
                continue
            r, c = self.rows(b), self.cols(b)
            sub = Ap[r["offset"]:r["offset"] + r["size"], c["offset"]:c["offset"] + c["size"]]
            if blk["kind"] == DENSE:
                self.D[b] = sub.toarray()
            else:
                dense = sub.toarray()
                nz = np.nonzero(np.any(dense != 0.0, axis=1))[0]
                X = np.zeros((r["size"], len(nz)))
                X[nz, np.arange(len(nz))] = 1.0
                self.X[b] = X
                self.Y[b] = dense[nz].T.copy()

    def to_dense(self, b=0):
        r, c = self.rows(b), self.cols(b)
        out = np.zeros((r["size"], c["size"]), self.dtype)
        k = self.kind(b)
        if k == DENSE:
            out[:] = self.D[b]
        elif k == ADM:
            out[:] = self.X[b] @ self.Y[b].T
        else:
            for s in self.bl[b]["sons"]:
                rs, cs = self.rows(s), self.cols(s)
                i0, j0 = rs["offset"] - r["offset"], cs["offset"] - c["offset"]
                out[i0:i0 + rs["size"], j0:j0 + cs["size"]] = self.to_dense(s)
        return out

    # ---- H-matrix times dense multivector --------------------------------
    def hmul(self, b, V):
        """block b (tau x sigma) times V (|sigma| x k)."""
        k = self.kind(b)
        if k == DENSE:
            return self.D[b] @ V
        if k == ADM:
            return self.X[b] @ (self.Y[b].T @ V)
        r, c = self.rows(b), self.cols(b)
        out = np.zeros((r["size"], V.shape[1]), np.result_type(self.dtype, V))
        for s in self.bl[b]["sons"]:
            rs, cs = self.rows(s), self.cols(s)
            i0, j0 = rs["offset"] - r["offset"], cs["offset"] - c["offset"]
            out[i0:i0 + rs["size"]] += self.hmul(s, V[j0:j0 + cs["size"]])
        return out

    def hmulT(self, b, V):
        """transpose of block b (sigma x tau) times V (|tau| x k)."""
        k = self.kind(b)
        if k == DENSE:
            return self.D[b].T @ V
        if k == ADM:
            return self.Y[b] @ (self.X[b].T @ V)
        r, c = self.rows(b), self.cols(b)
        out = np.zeros((c["size"], V.shape[1]), np.result_type(self.dtype, V))
        for s in self.bl[b]["sons"]:
            rs, cs = self.rows(s), self.cols(s)
            i0, j0 = rs["offset"] - r["offset"], cs["offset"] - c["offset"]
            out[j0:j0 + cs["size"]] += self.hmulT(s, V[i0:i0 + rs["size"]])
        return out

    # ---- triangular solves with a factored diagonal block ----------------
    def solve_lower(self, d, V):
        """Z = L_d^-1 P_d V (L unit lower, P the leaf pivots)."""
        if self.kind(d) == DENSE:
            Z = V[self.piv[d]]
            return sla.solve_triangular(self.D[d], Z, lower=True, unit_diagonal=True)
        n0 = self.split_rows(d)
        Z0 = self.solve_lower(self.son(d, 0, 0), V[:n0])
        V1 = V[n0:] - self.hmul(self.son(d, 1, 0), Z0)
        Z1 = self.solve_lower(self.son(d, 1, 1), V1)
        return np.vstack([Z0, Z1])

    def solve_upper(self, d, V):
        """Z = U_d^-1 V."""
        if self.kind(d) == DENSE:
            return sla.solve_triangular(self.D[d], V, lower=False)
        n0 = self.split_rows(d)
        Z1 = self.solve_upper(self.son(d, 1, 1), V[n0:])
        V0 = V[:n0] - self.hmul(self.son(d, 0, 1), Z1)
        Z0 = self.solve_upper(self.son(d, 0, 0), V0)
        return np.vstack([Z0, Z1])

    def solve_upperT(self, d, W):
        """Z = U_d^-T W (used for B <- B U^-1 as B^T <- U^-T B^T)."""
        if self.kind(d) == DENSE:
            return sla.solve_triangular(self.D[d], W, lower=False, trans="T")
        n0 = self.split_rows(d)
        Z0 = self.solve_upperT(self.son(d, 0, 0), W[:n0])
        W1 = W[n0:] - self.hmulT(self.son(d, 0, 1), Z0)
        Z1 = self.solve_upperT(self.son(d, 1, 1), W1)
        return np.vstack([Z0, Z1])

    # ---- H-trsm ------------------------------------------------------------
    def trsm_left(self, d, b):
        """b <- L_d^-1 P_d b (block row of the diagonal block d)."""
        k = self.kind(b)
        if k == ADM:
            self.X[b] = self.solve_lower(d, self.X[b])
        elif k == DENSE:
            self.D[b] = self.solve_lower(d, self.D[b])
        else:
            for j in range(2):
                self.trsm_left(self.son(d, 0, 0), self.son(b, 0, j))
                self.gemm(self.son(b, 1, j), self.son(d, 1, 0), self.son(b, 0, j))
                self.trsm_left(self.son(d, 1, 1), self.son(b, 1, j))

    def trsm_right(self, b, d):
        """b <- b U_d^-1 (block column of the diagonal block d)."""
        k = self.kind(b)
        if k == ADM:
            self.Y[b] = self.solve_upperT(d, self.Y[b])
        elif k == DENSE:
            self.D[b] = self.solve_upperT(d, self.D[b].T).T
        else:
            for i in range(2):
                self.trsm_right(self.son(b, i, 0), self.son(d, 0, 0))
                self.gemm(self.son(b, i, 1), self.son(b, i, 0), self.son(d, 0, 1))
                self.trsm_right(self.son(b, i, 1), self.son(d, 1, 1))

    # ---- H-gemm: c <- c - a b -----------------------------------------------
    def product(self, a, b):
        """Low-rank factors (X, Y) with X Y^T = a b (truncated only when both
        operands are subdivided)."""
        ka, kb = self.kind(a), self.kind(b)
        if ka == ADM:
            return self.X[a], self.hmulT(b, self.Y[a])
        if kb == ADM:
            return self.hmul(a, self.X[b]), self.Y[b]
        if ka == DENSE and kb == DENSE:
            return self.D[a], self.D[b].T
        if ka == DENSE:  # row cluster of a is a leaf
            return np.eye(self.rows(a)["size"]), self.hmulT(b, self.D[a].T)
        if kb == DENSE:  # column cluster of b is a leaf
            return self.hmul(a, self.D[b]), np.eye(self.cols(b)["size"])
        # both subdivided: son products, each summed and truncated, then agglomerated
        m0, n0 = self.split_rows(a), self.split_cols(b)
        m, n = self.rows(a)["size"], self.cols(b)["size"]
        Xs, Ys = [], []
        for i in range(2):
            for j in range(2):
                px, py = [], []
                for k in range(2):
                    x, y = self.product(self.son(a, i, k), self.son(b, k, j))
                    px.append(x)
                    py.append(y)
                x, y = truncate(np.hstack(px), np.hstack(py), self.eps)
                X = np.zeros((m, x.shape[1]), x.dtype)
                Y = np.zeros((n, x.shape[1]), y.dtype)
                if i == 0:
                    X[:m0] = x
                else:
                    X[m0:] = x
                if j == 0:
                    Y[:n0] = y
                else:
                    Y[n0:] = y
                Xs.append(X)
                Ys.append(Y)
        return truncate(np.hstack(Xs), np.hstack(Ys), self.eps)

    def add_lr(self, c, X, Y):
        """c <- c + X Y^T in the format of c (truncated in low-rank leaves)."""
        k = self.kind(c)
        if k == DENSE:
            self.D[c] = self.D[c] + X @ Y.T
        elif k == ADM:
            self.X[c], self.Y[c] = truncate(np.hstack([self.X[c], X]),
                                            np.hstack([self.Y[c], Y]), self.eps)
        else:
            m0, n0 = self.split_rows(c), self.split_cols(c)
            for i in range(2):
                for j in range(2):
                    xs = X[:m0] if i == 0 else X[m0:]
                    ys = Y[:n0] if j == 0 else Y[n0:]
                    self.add_lr(self.son(c, i, j), xs, ys)

    def gemm(self, c, a, b):
        if self.kind(c) == SUB and self.kind(a) == SUB and self.kind(b) == SUB:
            for i in range(2):
                for j in range(2):
                    for k in range(2):
                        self.gemm(self.son(c, i, j), self.son(a, i, k), self.son(b, k, j))
            return
        X, Y = self.product(a, b)
        self.add_lr(c, -X, Y)

    # ---- H-LU (Alg. 1 step II) -------------------------------------------
    def lu(self, d=0):
        if self.kind(d) == DENSE:
            self.D[d], self.piv[d] = getrf(self.D[d])
            return
        d00, d01 = self.son(d, 0, 0), self.son(d, 0, 1)
        d10, d11 = self.son(d, 1, 0), self.son(d, 1, 1)
        self.lu(d00)
        self.trsm_left(d00, d01)
        self.trsm_right(d10, d00)
        self.gemm(d11, d10, d01)
        self.lu(d11)

    # ---- preconditioner application (Alg. 1 step III) --------------------
    def solve(self, r):
        """(LU)_H^-1 r in the permuted order; r (N,) or (N, k)."""
        V = r.reshape(r.shape[0], -1)
        Z = self.solve_upper(0, self.solve_lower(0, V))
        return Z.reshape(r.shape)

    # ---- statistics ---------------------------------------------------------
    def ranks(self):
        return {b: self.X[b].shape[1] for b in self.X}

    def storage_words(self):
        w = sum(d.size for d in self.D.values())
        w += sum(self.X[b].size + self.Y[b].size for b in self.X)
        return w


class HLUPreconditioner:
    """Alg. 1 I-II for a CSR matrix A: permute, fill A_H, factor.  apply(r)
    returns (LU)_H^-1 r in the original DOF order."""

    def __init__(self, A, perm, clusters, blocks, eps):
        self.perm = np.asarray(perm, dtype=np.int64)
        Ap = A[self.perm][:, self.perm].tocsr()
        self.H = HMatrix(clusters, blocks, eps)
        self.H.fill(Ap)
        self.H.lu(0)

    def apply(self, r):
        rp = r[self.perm]
        zp = self.H.solve(rp)
        z = np.empty_like(zp)
        z[self.perm] = zp
        return z

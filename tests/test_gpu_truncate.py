"""GPU parity of the recompression kernel on its own (one TK_TRUNC task run by
the device executor through hlu_debug_truncate) against the oracle's
truncation (Sec. 4 truncated SVD: QR of both factors, SVD of the core, keep
s_i > eps s_1).

Inputs have a prescribed spectrum with a clear gap at eps, so the kept rank
is unique: X Y^T = U diag(s) V^T is handed over as X = U diag(s) M and
Y = V M^-T with a random well-conditioned M, so neither stack is
orthogonal.  The shapes reach every route of the kernel: the stack held in
shared memory (one compression), the stack in global scratch with its
piecewise compressions, and (FP32) the dense sum for targets up to 128 x 128.
"""
import numpy as np
import pytest

from oracle import hmatrix

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


def stack(m, n, w, r_keep, eps, seed):
    """X (m x w), Y (n x w) with X Y^T of singular values: r_keep values in
    [20 eps, 1], then the rest at or below eps / 20."""
    rng = np.random.default_rng(seed)
    k = min(w, m, n)
    s = np.concatenate([np.logspace(0, np.log10(20 * eps), r_keep),
                        np.logspace(np.log10(eps / 20), np.log10(eps / 1e4), k - r_keep)])
    U = np.linalg.qr(rng.standard_normal((m, k)))[0]
    V = np.linalg.qr(rng.standard_normal((n, k)))[0]
    M = np.linalg.qr(rng.standard_normal((k, w)).T)[0].T  # k x w, orthonormal rows
    M = M * rng.uniform(0.5, 2.0, size=(1, w))
    X = (U * s) @ M
    # Y with X Y^T = U diag(s) V^T: Y^T = pinv(M) V^T (M has full row rank)
    Y = (np.linalg.pinv(M) @ V.T).T
    return X, Y, s


def quadrant_stack(m, n, wq, eps, seed, npieces=4):
    """npieces pieces of wq columns, piece q nonzero only in quadrant
    ((q mod 4) // 2, q mod 2) of the m x n target (rows split at m // 2,
    columns at n // 2)."""
    rng = np.random.default_rng(seed)
    mh, nh = m // 2, n // 2
    X = np.zeros((m, npieces * wq))
    Y = np.zeros((n, npieces * wq))
    for q in range(npieces):
        i, j = (q % 4) // 2, q % 2
        r0, r1 = (0, mh) if i == 0 else (mh, m)
        c0, c1 = (0, nh) if j == 0 else (nh, n)
        s = np.logspace(0, np.log10(eps / 1e3), wq) * (1.0 + q)
        X[r0:r1, q * wq:(q + 1) * wq] = rng.standard_normal((r1 - r0, wq)) * s
        Y[c0:c1, q * wq:(q + 1) * wq] = rng.standard_normal((c1 - c0, wq))
    return X, Y


GENERIC = [
    # (m, n, wq or w, pieces of, flags, eps): bounds only (no designed gap);
    # flag 8 (test only): eight quadrant pieces instead of four
    (120, 110, 20, 20, 4, 1e-4),    # four quadrant pieces (an agglomeration)
    (150, 140, 12, 12, 4, 1e-6),
    (200, 180, 16, 16, 4, 1e-6),
    (100, 66, 5, 5, 4 | 8, 1e-6),   # eight pieces, two per quadrant
    (128, 100, 8, 8, 4 | 8, 1e-6),
    (300, 260, 24, 24, 4, 1e-6),
    (64, 64, 30, 30, 4, 1e-5),
    (5, 3, 8, 4, 0, 1e-4),          # tiny targets
    (1, 40, 4, 0, 0, 1e-4),
    (16, 2, 10, 5, 2, 1e-4),        # transposed Y views
    (70, 80, 50, 10, 1, 1e-4),      # the target is the first piece
    (200, 30, 40, 10, 1, 1e-6),     # m > w > n
    (373, 390, 5, 3, 0, 1e-6),      # long stacks in shared memory
    (373, 390, 10, 5, 1, 1e-6),
    (410, 357, 6, 6, 4, 1e-6),      # quadrants, long stacks
    (300, 280, 21, 11, 2, 1e-6),
    (25, 180, 44, 11, 0, 1e-6),     # n > w > m
    (150, 120, 40, 20, 16, 1e-6),   # flag 16 (test only): the two pieces are equal (rank deficient)
    (100, 64, 64, 64, 32, 1e-6),    # flag 32 (test only): one piece is an identity factor
    (90, 100, 60, 20, 3, 1e-6),     # both
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m,n,w,pw,flags,eps", GENERIC)
def test_truncation_bounds(hlu, prec, m, n, w, pw, flags, eps):
    """The kept factors are an eps-truncation: ||F - X Y^T|| <= eps s_1 (plus
    rounding), the same operator as the oracle's up to the values at the
    threshold, and the rank within two of the oracle's."""
    rng = np.random.default_rng(m * 31 + n * 7 + w + flags)
    if flags & 4:
        X, Y = quadrant_stack(m, n, w, eps, seed=m + n + w, npieces=8 if flags & 8 else 4)
        flags &= 7
    else:
        X = rng.standard_normal((m, w)) * np.logspace(0, np.log10(eps / 1e3), w)
        Y = rng.standard_normal((n, w))
        if flags & 16:  # second half repeats the first: exactly rank deficient
            X[:, w // 2:] = X[:, :w // 2]
            Y[:, w // 2:] = -0.5 * Y[:, :w // 2]
        if flags & 32:  # Y = I on the first n rows (a dense block as X, identity as Y)
            X = rng.standard_normal((m, w)) * np.logspace(0, np.log10(eps / 1e3), w)[None, :]
            Y = np.eye(n, w)
        flags &= 7
    F = X @ Y.T
    s = np.linalg.svd(F, compute_uv=False)
    Xo, Yo = hmatrix.truncate(X, Y, eps)
    P = hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32
    cap = min(64, m, n)
    Xd, Yd, st = hlu.debug_truncate(X, Y, eps, cap=cap, precision=P, piece_cols=pw, flags=flags)
    assert st[0] == 0
    r = Xd.shape[1]
    if prec == "fp64" or eps >= 1e-5:  # below that FP32 cannot place the threshold
        assert abs(r - min(Xo.shape[1], cap)) <= 2, (r, Xo.shape[1])
    rnd = 1e-12 if prec == "fp64" else 3e-6 * np.linalg.norm(X, 2) * np.linalg.norm(Y, 2) / s[0]
    assert np.linalg.norm(F - Xd @ Yd.T, 2) <= (1.05 * eps + rnd) * s[0]
    if r:
        assert np.linalg.norm(Yd.T @ Yd - np.eye(r), 2) <= (1e-12 if prec == "fp64" else 1e-5)


CASES = [
    # (m, n, w, pieces of, kept rank, eps)
    (60, 70, 30, 0, 12, 1e-4),       # shared-memory stack
    (100, 90, 40, 16, 20, 1e-6),     # shared-memory stack, three pieces
    (30, 20, 40, 0, 8, 1e-4),        # wider than tall
    (128, 128, 48, 24, 30, 1e-6),
    (600, 500, 80, 40, 25, 1e-4),    # global scratch
    (1500, 1400, 200, 64, 40, 1e-5),  # piecewise compressions
    (100, 120, 90, 30, 35, 1e-4),    # FP32: dense sum route
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m,n,w,pw,rk,eps", CASES)
def test_truncation_matches_oracle(hlu, prec, m, n, w, pw, rk, eps):
    X, Y, s = stack(m, n, w, rk, eps, seed=m + 7 * n + w)
    Xo, Yo = hmatrix.truncate(X, Y, eps)
    assert Xo.shape[1] == rk  # the oracle sees the designed gap
    P = hlu.HLU_FP64 if prec == "fp64" else hlu.HLU_FP32
    Xd, Yd, st = hlu.debug_truncate(X, Y, eps, cap=min(64, m, n), precision=P, piece_cols=pw)
    assert st[0] == 0 and st[2] == 0
    assert Xd.shape[1] == rk
    F = Xo @ Yo.T
    tol = 1e-9 if prec == "fp64" else 2e-4
    # the same truncated operator as the oracle's, to rounding (and to the
    # dropped tail, which is below eps / 20 of s_1)
    err = np.linalg.norm(Xd @ Yd.T - F, 2) / s[0]
    assert err <= tol + 0.1 * eps, err
    assert np.linalg.norm(Yd.T @ Yd - np.eye(rk), 2) <= (1e-12 if prec == "fp64" else 1e-5)

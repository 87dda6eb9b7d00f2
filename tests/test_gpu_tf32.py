"""The TF32 tensor-core path (HLU_TF32, tcgen05 MMAs with the accumulator in
tensor memory, each operand split into TF32 high and low parts) through the
C ABI.  The tile product on its own equals the split product up to FP32
accumulation; factorisations whose tile products run on the tensor cores
meet the oracle's operator-error bar and stay close to the FP32 path, and
FGMRES brings their solutions to 1e-7 of the direct solve."""
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


def tf32_round(x):
    """Nearest TF32 value (10 stored mantissa bits), ties away from zero, as
    float32: add half of the dropped 13 bits to the magnitude, then clear them."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    mag = (u & 0x7FFFFFFF) + 0x1000
    out = (u & 0x80000000) | (mag & 0x7FFFE000)
    return out.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("K", [1, 5, 32, 33, 100, 256])
def test_tf32_tile_product(hlu, K):
    """D = A B from the tensor cores with each operand split into a TF32 part
    and the TF32 rounding of its remainder: D equals
    A_hi B_hi + A_hi B_lo + A_lo B_hi up to FP32 accumulation, and A B (the
    FP32 product) to about 2^-21 relative, far closer than the plain TF32
    product A_hi B_hi."""
    import ctypes
    rng = np.random.default_rng(K)
    A = rng.standard_normal((64, K)).astype(np.float32)
    B = rng.standard_normal((K, 64)).astype(np.float32)
    dA = torch.from_numpy(np.asfortranarray(A).ravel(order="F")).cuda()
    dB = torch.from_numpy(np.asfortranarray(B).ravel(order="F")).cuda()
    dD = torch.zeros(64 * 64, dtype=torch.float32, device="cuda")
    st = (ctypes.c_int32 * 1)()
    rc = hlu.lib().hlu_debug_tf32_tile(ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                                        ctypes.c_void_p(dD.data_ptr()), K, st)
    assert rc == 0 and st[0] == 0
    D = dD.cpu().numpy().reshape(64, 64, order="F").astype(np.float64)
    Ah, Bh = tf32_round(A), tf32_round(B)
    Al, Bl = tf32_round(A - Ah), tf32_round(B - Bh)  # A - A_hi is exact in FP32
    Ah, Bh, Al, Bl = (x.astype(np.float64) for x in (Ah, Bh, Al, Bl))
    ref = Ah @ Bh + Ah @ Bl + Al @ Bh
    scale = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    # the partial products are exact in FP32; only the FP32 accumulation rounds
    assert np.all(np.abs(D - ref) <= (K + 2) * 2.0 ** -23 * scale + 1e-30)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    assert np.all(np.abs(D - exact) <= (K + 4) * 2.0 ** -21 * scale + 1e-30)
    if K >= 32:  # the split matters: the plain TF32 product is much further off
        assert np.abs(Ah @ Bh - exact).max() > 16 * np.abs(D - exact).max()


def _op_error(apply, A, nvec=3, seed=11):
    N = A.shape[0]
    Z = np.stack([synth.normal(seed + i, N) for i in range(nvec)], axis=1)
    E = Z - apply(A @ Z)
    return max(np.linalg.norm(E[:, i]) / np.linalg.norm(Z[:, i]) for i in range(nvec))


def _gpu_apply(hlu, h, X):
    N = X.shape[0]
    b = hlu.colmajor(N, X.shape[1])
    b.copy_(torch.from_numpy(np.asfortranarray(X)))
    x = hlu.colmajor(N, X.shape[1])
    hlu.hlu_solve(h, b, x)
    torch.cuda.synchronize()
    return x.cpu().numpy()


@pytest.mark.parametrize("n,kappa,eps", [(6, 4.0, 1e-2), (8, 8.0, 1e-3), (10, 6.0, 1e-4)])
def test_tf32_factor_within_2x_of_oracle(hlu, n, kappa, eps):
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    perm, cl, bl = trees.build_trees(m, 32, 2.0)
    e_or = _op_error(hmatrix.HLUPreconditioner(A, perm, cl, bl, eps).apply, A)
    h = hlu.hlu_build(n, kappa, 32, 2.0, eps)
    try:
        hlu.hlu_factor(h, hlu.HLU_TF32)
        info = hlu.hlu_factor_stats(h)
        assert info["rank_cap_hits"] == 0
        e_tf = _op_error(lambda R: _gpu_apply(hlu, h, R), A)
        assert e_tf <= 2.0 * e_or, (e_tf, e_or)
        # the FP32 path on the same handle gives a comparable preconditioner
        hlu.hlu_factor(h, hlu.HLU_FP32)
        e_32 = _op_error(lambda R: _gpu_apply(hlu, h, R), A)
        assert e_tf <= 1.5 * e_32, (e_tf, e_32)
    finally:
        hlu.hlu_destroy(h)


def test_tf32_factor_fgmres_to_1e7(hlu):
    """FP64 flexible GMRES recovers full accuracy from the TF32 factor."""
    n, kappa = 8, 8.0
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsc()
    N = A.shape[0]
    B = np.stack([synth.normal(synth.rhs_seed(2, 9, j), N) for j in range(3)], axis=1)
    xs = spla.splu(A).solve(B)
    h = hlu.hlu_build(n, kappa, 32, 2.0, 1e-4)
    try:
        hlu.hlu_factor(h, hlu.HLU_TF32)
        b = hlu.colmajor(N, 3)
        b.copy_(torch.from_numpy(np.asfortranarray(B)))
        x = hlu.colmajor(N, 3)
        st = hlu.gmres_solve(h, b, x, restart=50, tol=1e-10, maxit=500)
        torch.cuda.synchronize()
        assert st["converged"] == 1
        xg = x.cpu().numpy()
        for j in range(3):
            assert np.linalg.norm(xg[:, j] - xs[:, j]) <= 1e-7 * np.linalg.norm(xs[:, j]), j
    finally:
        hlu.hlu_destroy(h)

"""Pins of the oracle's complex path (no GPU): the time-harmonic operator
with conductivity, curl(beta^-1 curl E) - kappa E with
kappa = omega^2 (alpha + i chi / omega) (Sec. 2), complex H-matrix blocks
X Y^T with complex factors (Definition 1), the H-LU in complex arithmetic
and Algorithm 1's Richardson iteration on it.

What fixes the answers here is not the oracle itself: a discrete cavity mode
from scipy's generalised eigensolver (A v = -i omega chi M v exactly at
resonance), the energy identity of a complex symmetric system with real
symmetric K and M, the reduction to the real assembly at chi = 0, LAPACK's
complex LU, prescribed complex singular value decompositions and the dense
complex solve.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import fem as F
from oracle import hmatrix as H
from oracle import krylov as K
from oracle import mesh as M
from oracle import trees as T


def _cgauss(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_reduces_to_the_real_assembly_without_conductivity():
    m = M.interior_edges(4)
    for omega, alpha in [(3.0, 1.0), (2.5, 1.7)]:
        Ac = F.assemble_time_harmonic(m, omega, alpha, 0.0)
        Ar = F.assemble(m, omega * np.sqrt(alpha))
        assert np.array_equal(Ac.indptr, Ar.indptr) and np.array_equal(Ac.indices, Ar.indices)
        assert np.all(Ac.data.imag == 0.0)
        assert np.abs(Ac.data.real - Ar.data).max() <= 1e-13 * np.abs(Ar.data).max()


def test_complex_symmetric_not_hermitian():
    m = M.interior_edges(3)
    A = F.assemble_time_harmonic(m, 2.0, 1.0, 0.4).toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()  # summation order only
    assert np.abs(A - A.conj().T).max() > 1e-3 * np.abs(A).max()
    assert np.all(A.diagonal().imag < 0)  # -omega chi M_ii, M SPD


def test_resonance_mode_is_damped_by_conductivity_alone():
    """K v = lambda M v (scipy's generalised eigensolver): at omega^2 alpha =
    lambda the real operator annihilates v, and with chi > 0 A v is exactly
    -i omega chi M v."""
    m = M.interior_edges(4)
    Ks, Ms = F.assemble(m, 0.0, parts=True)
    Kd, Md = Ks.toarray(), Ms.toarray()
    lam, vecs = sla.eigh(Kd, Md)
    nul = (4 - 1) ** 3  # gradients: the kernel of K
    assert np.all(np.abs(lam[:nul]) < 1e-8 * lam[-1]) and lam[nul] > 1.0
    lam1, v = lam[nul], vecs[:, nul]
    alpha, chi = 1.3, 0.25
    omega = np.sqrt(lam1 / alpha)
    A0 = F.assemble_time_harmonic(m, omega, alpha, 0.0)
    assert np.linalg.norm(A0 @ v) <= 1e-9 * np.linalg.norm(Kd @ v)
    A = F.assemble_time_harmonic(m, omega, alpha, chi)
    want = -1j * omega * chi * (Md @ v)
    assert np.linalg.norm(A @ v - want) <= 1e-9 * np.linalg.norm(want)
    # nonsingular: the mode is solvable with conductivity
    x = spla.spsolve(A.tocsc(), Md @ v)
    assert np.linalg.norm(A @ x - Md @ v) <= 1e-10 * np.linalg.norm(Md @ v)


@pytest.mark.parametrize("omega,alpha,chi", [(3.0, 1.0, 0.7), (5.0, 2.0, 3.0)])
def test_energy_identity(omega, alpha, chi):
    """A x = b with A = K - (omega^2 alpha + i omega chi) M, K and M real
    symmetric: x^H b = x^H K x - omega^2 alpha x^H M x - i omega chi x^H M x."""
    m = M.interior_edges(4)
    Ks, Ms = F.assemble(m, 0.0, parts=True)
    A = F.assemble_time_harmonic(m, omega, alpha, chi)
    rng = np.random.default_rng(11)
    b = _cgauss(rng, A.shape[0])
    x = spla.spsolve(A.tocsc(), b)
    xk = np.vdot(x, Ks @ x)
    xm = np.vdot(x, Ms @ x)
    assert abs(xk.imag) <= 1e-12 * abs(xk) and abs(xm.imag) <= 1e-12 * abs(xm)
    lhs = np.vdot(x, b)
    rhs = xk.real - omega ** 2 * alpha * xm.real - 1j * omega * chi * xm.real
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_complex_getrf_matches_lapack():
    rng = np.random.default_rng(5)
    for n in (1, 6, 32):
        A = _cgauss(rng, n, n)
        LU, p = H.getrf(A)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        P, L2, U2 = sla.lu(A)  # A = P L U, pivot on |a|
        assert np.allclose(L @ U, A[p], atol=1e-12)
        assert np.allclose(L, L2, atol=1e-12) and np.allclose(U, U2, atol=1e-12)


def test_complex_truncation_known_singular_values():
    rng = np.random.default_rng(2)
    m, n = 50, 40
    U, _ = np.linalg.qr(_cgauss(rng, m, 5))
    V, _ = np.linalg.qr(_cgauss(rng, n, 5))
    s = np.array([2.0, 0.5, 1e-2, 3e-5, 1e-9])
    F_ = (U * s) @ V.T  # X Y^T form with complex factors
    # a redundant stack: the product plus a zero contribution
    X = np.hstack([U * s, _cgauss(rng, m, 3)])
    Y = np.hstack([V, np.zeros((n, 3))])
    for eps, r in [(1e-1, 2), (1e-3, 3), (1e-6, 4), (1e-12, 5)]:
        Xt, Yt = H.truncate(X, Y, eps)
        assert Xt.shape[1] == r and Xt.dtype == np.complex128
        err = np.linalg.norm(F_ - Xt @ Yt.T, 2)
        tail = s[r] if r < len(s) else 0.0
        assert abs(err - tail) <= 1e-12 * s[0]
    Xz, Yz = H.truncate(np.zeros((4, 2), complex), np.ones((3, 2), complex), 1e-4)
    assert Xz.shape == (4, 0) and Yz.shape == (3, 0) and Xz.dtype == np.complex128


def _complex_problem(n, omega, chi, leaf, beta=None):
    m = M.interior_edges(n)
    A = F.assemble_time_harmonic(m, omega, 1.0, chi, beta=beta)
    perm, cl, bl = T.build_trees(m, leaf, 2.0)
    return m, A, perm, cl, bl


@pytest.mark.parametrize("n,omega,chi,leaf", [(4, 2.0, 0.5, 16), (5, 4.0, 2.0, 32)])
def test_complex_hlu_tight_eps_is_dense_solve(n, omega, chi, leaf):
    m, A, perm, cl, bl = _complex_problem(n, omega, chi, leaf)
    P = H.HLUPreconditioner(A, perm, cl, bl, 1e-14)
    rng = np.random.default_rng(9)
    b = _cgauss(rng, A.shape[0])
    x = np.linalg.solve(A.toarray(), b)
    z = P.apply(b)
    assert z.dtype == np.complex128
    assert np.linalg.norm(z - x) <= 1e-9 * np.linalg.norm(x)


def test_complex_hlu_error_falls_with_eps():
    m, A, perm, cl, bl = _complex_problem(5, 3.0, 1.0, 32)
    Ad = A.toarray()
    N = Ad.shape[0]
    errs = []
    for eps in (1e-1, 1e-2, 1e-4, 1e-6):
        P = H.HLUPreconditioner(A, perm, cl, bl, eps)
        errs.append(np.linalg.norm(np.eye(N) - P.apply(Ad), 2))
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[-1] < 1e-3


def test_complex_richardson_reaches_the_direct_solve():
    """Algorithm 1 (H-LU at eps 1e-4, Richardson to TOL 1e-8) on Example 3's
    magnet with conductivity: the paper's complex kappa, the magnet's beta,
    J_S = [10, 10, 10]^T."""
    n = 6
    m = M.interior_edges(n)
    beta = F.magnet_beta(m, 10.0)
    _, A, perm, cl, bl = _complex_problem(n, np.sqrt(10.0), 0.5, 32, beta=beta)
    b = F.constant_current_rhs(m, (10.0, 10.0, 10.0)).astype(complex)
    P = H.HLUPreconditioner(A, perm, cl, bl, 1e-4)
    x, info = K.richardson(lambda v: A @ v, b, P.apply, tol=1e-8)
    assert info["history"][-1] < 1e-8 and info["iters"] <= 10
    xs = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)
    assert np.abs(xs.imag).max() > 1e-3 * np.abs(xs).max()  # the damping is felt


def test_complex_fgmres_textbook_cases():
    """A diagonal matrix with m distinct complex eigenvalues is solved in m
    steps (its Krylov space has dimension m); an exact preconditioner in one;
    a random complex system to the tolerance of numpy's dense solve."""
    rng = np.random.default_rng(4)
    lam = np.array([2.0 + 1j, -1.0 + 0.5j, 3.0 - 2j, 0.5 + 4j, -2.0 - 1j])
    d = np.repeat(lam, 8)
    b = _cgauss(rng, d.shape[0])
    x, info = K.fgmres(lambda v: d * v, b, restart=20, tol=1e-12)
    assert info["converged"] and info["iters"] <= 5, info["iters"]
    assert np.linalg.norm(x - b / d) <= 1e-10 * np.linalg.norm(b / d)
    A = _cgauss(rng, 40, 40) + 20 * np.eye(40)  # spectrum in a disk of radius ~9 around 20
    b = _cgauss(rng, 40)
    Ainv = np.linalg.inv(A)
    x, info = K.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, restart=10, tol=1e-12)
    assert info["converged"] and info["iters"] == 1
    x, info = K.fgmres(lambda v: A @ v, b, restart=8, tol=1e-11)
    xs = np.linalg.solve(A, b)
    assert info["converged"] and np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b) * 1.0001


def test_complex_fgmres_with_the_complex_hlu():
    """FGMRES with the complex H-LU on the conducting magnet reaches the direct
    solve, in no more steps than Algorithm 1's Richardson iteration."""
    n = 6
    m = M.interior_edges(n)
    beta = F.magnet_beta(m, 10.0)
    _, A, perm, cl, bl = _complex_problem(n, np.sqrt(10.0), 0.5, 32, beta=beta)
    b = F.constant_current_rhs(m, (10.0, 10.0, 10.0)).astype(complex)
    P = H.HLUPreconditioner(A, perm, cl, bl, 1e-4)
    x, info = K.fgmres(lambda v: A @ v, b, P.apply, restart=30, tol=1e-10)
    xs = spla.spsolve(A.tocsc(), b)
    assert info["converged"] and np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)
    _, rinfo = K.richardson(lambda v: A @ v, b, P.apply, tol=1e-10)
    assert info["iters"] <= rinfo["iters"], (info["iters"], rinfo["iters"])


def test_real_fgmres_is_unchanged_by_the_complex_path():
    """Real input keeps real arrays and the real rotations."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 30)) + 12 * np.eye(30)
    b = rng.standard_normal(30)
    x, info = K.fgmres(lambda v: A @ v, b, restart=6, tol=1e-12)
    assert x.dtype == np.float64 and info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)

"""Pins of the oracle's GMRES / FGMRES and Richardson loop (no GPU)."""
import numpy as np

from oracle import krylov as K


def test_gmres_diagonal_distinct_eigenvalues():
    # a diagonal matrix with m distinct eigenvalues: GMRES terminates in <= m steps
    rng = np.random.default_rng(0)
    ev = np.array([1.0, 2.0, 3.5, 7.0, 11.0])
    d = ev[rng.integers(0, len(ev), 200)]
    b = rng.standard_normal(200)
    x, info = K.fgmres(lambda v: d * v, b, restart=50, tol=1e-12)
    assert info["converged"] and info["iters"] <= 5
    assert np.allclose(x, b / d, rtol=1e-9)


def test_exact_preconditioner_one_step():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 40)) + 40 * np.eye(40)
    b = rng.standard_normal(40)
    x, info = K.fgmres(lambda v: A @ v, b, precond=lambda v: np.linalg.solve(A, v), tol=1e-10)
    assert info["iters"] == 1 and info["converged"]


def test_nonsymmetric_with_restart():
    rng = np.random.default_rng(2)
    n = 120
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, info = K.fgmres(lambda v: A @ v, b, restart=5, tol=1e-10, maxit=2000)
    assert info["converged"] and info["restarts"] > 1
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.0001
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-7)


def test_flexible_varying_preconditioner():
    rng = np.random.default_rng(3)
    n = 60
    A = np.diag(np.linspace(1, 50, n)) + 0.1 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    calls = [0]
    Ainv = np.linalg.inv(A)

    def prec(v):  # a different (inexact) preconditioner each call
        calls[0] += 1
        noise = 0.05 * rng.standard_normal((n, n)) / np.sqrt(n) / 50.0
        return (Ainv + noise) @ v

    x, info = K.fgmres(lambda v: A @ v, b, precond=prec, tol=1e-11)
    assert info["converged"]
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b) * 1.0001


def test_richardson_exact_preconditioner():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 30)) + 30 * np.eye(30)
    b = rng.standard_normal(30)
    x, info = K.richardson(lambda v: A @ v, b, lambda v: np.linalg.solve(A, v), tol=1e-8)
    assert info["iters"] == 2 and info["history"][0] == 1.0
    assert info["error"] < 1e-10


def test_zero_rhs():
    x, info = K.fgmres(lambda v: v, np.zeros(5))
    assert info["converged"] and not x.any()

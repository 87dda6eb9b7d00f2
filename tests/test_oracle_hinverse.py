"""Pins of the oracle's Schulz H-inverse (no GPU): against the exact inverse,
the Schulz iteration's convergence law and the truncation tolerance."""
import numpy as np
import pytest

from oracle import fem, hinverse, mesh, trees


def _problem(n, kappa, leaf=8):
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    perm, cl, bl = trees.build_trees(m, leaf, 2.0)
    return A, perm, cl, bl


def test_tight_eps_gives_the_exact_inverse():
    A, perm, cl, bl = _problem(3, 1.5)
    B, info = hinverse.schulz_inverse(A, perm, cl, bl, eps=1e-15, tol=1e-12, maxit=200)
    Ainv = np.linalg.inv(A.toarray())
    assert np.linalg.norm(B - Ainv, 2) <= 1e-9 * np.linalg.norm(Ainv, 2)
    assert info["residuals"][-1] <= 1e-12


def test_schulz_convergence_law():
    """||I - A X_0|| < 1 for the scaled start, and in exact arithmetic the
    residual matrix squares each step (R_{k+1} = R_k^2), so the norm at least
    squares once the block truncation is negligible."""
    A, perm, cl, bl = _problem(3, 2.0)
    _, info = hinverse.schulz_inverse(A, perm, cl, bl, eps=1e-15, tol=1e-13, maxit=200)
    r = info["residuals"]
    assert r[0] < 1.0
    assert all(b <= a * (1 + 1e-9) for a, b in zip(r, r[1:]))  # monotone
    for a, b in zip(r, r[1:]):
        if a < 0.5 and a > 1e-6:
            assert b <= a * a * (1 + 1e-6) + 1e-13, (a, b)


def test_alpha_is_the_inverse_of_the_one_and_inf_norms():
    A, perm, cl, bl = _problem(2, 1.0)
    _, info = hinverse.schulz_inverse(A, perm, cl, bl, eps=1e-12, tol=1e-8)
    Ad = A.toarray()
    assert info["alpha"] == pytest.approx(1.0 / (np.abs(Ad).sum(0).max() * np.abs(Ad).sum(1).max()))


def test_residual_falls_with_eps():
    A, perm, cl, bl = _problem(4, 3.0, leaf=16)
    finals = []
    for eps in (3e-2, 1e-2, 1e-4):
        _, info = hinverse.schulz_inverse(A, perm, cl, bl, eps=eps, tol=1e-12, maxit=80)
        finals.append(min(info["residuals"]))
    assert finals[0] > finals[1] > finals[2]

"""Restarted (flexible) GMRES with a right preconditioner, and the
preconditioned Richardson loop of Algorithm 1 (oracle; test infrastructure
only).

Paper: Sec. 4, Example 1 - preconditioned GMRES stopped at a relative residual
TOL, restarted after a fixed number of steps; Algorithm 1 step III
(r = b - A x, err = ||r|| / ||b||, x <- x + U^-1 (L^-1 r), stop when err < TOL) and
step IV (error = ||A x - b||_2).

Readings:
  * a complex system takes the Hermitian inner product and complex Givens
    rotations (the rotated column's subdiagonal entry is a norm, so the
    rotation's sine stays real);
  * right preconditioning: A M^-1 u = b, x = M^-1 u.  The flexible form stores
    z_j = M^-1 v_j and forms x = x0 + Z y, which also allows M to change between
    applications (an FP32 factor inside an FP64 Krylov loop);
  * x0 = 0; classical Gram-Schmidt applied twice (CGS2); Givens rotations on the
    Hessenberg matrix; stop when the rotated residual estimate falls to
    tol ||b||, then check the true residual ||b - A x|| and restart if it is not
    below tol ||b|| (up to maxit total inner steps).

Pins (tests/test_oracle_krylov.py): a diagonal matrix with m distinct
eigenvalues converges in m steps; the exact preconditioner M = A converges in
one step; the result solves random nonsymmetric systems to the tolerance;
Richardson with M = A stops after its first check.  Complex
(tests/test_oracle_complex.py): a diagonal matrix with m distinct complex
eigenvalues in m steps, an exact preconditioner in one, numpy's dense complex
solve, and the complex H-LU on the conducting magnet reaching the direct solve.
"""
import numpy as np


def fgmres(matvec, b, precond=None, restart=50, tol=1e-8, maxit=1000):
    """Returns (x, info) with info = dict(iters, restarts, converged, relres,
    history).  matvec(v) -> A v; precond(v) -> M^-1 v (identity if None).
    A complex system (the complex kappa of Sec. 2) uses the Hermitian inner
    product (h = V^H w) and complex Givens rotations; real input takes the
    real operations unchanged."""
    cplx = np.iscomplexobj(b)
    dt = np.complex128 if cplx else np.float64
    b = np.asarray(b, dtype=dt)
    N = b.shape[0]
    x = np.zeros(N, dt)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return x, {"iters": 0, "restarts": 0, "converged": True, "relres": 0.0, "history": hist}
    M = precond if precond is not None else (lambda v: v.copy())
    iters = 0
    restarts = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        relres = beta / bnorm
        hist.append(relres)
        if relres <= tol or iters >= maxit:
            return x, {"iters": iters, "restarts": restarts, "converged": relres <= tol,
                       "relres": relres, "history": hist}
        m = restart
        V = np.zeros((N, m + 1), dt)
        Z = np.zeros((N, m), dt)
        Hm = np.zeros((m + 1, m), dt)
        cs = np.zeros(m, dt)
        sn = np.zeros(m)  # real: the subdiagonal entry being annihilated is a norm
        g = np.zeros(m + 1, dt)
        g[0] = beta
        V[:, 0] = r / beta
        j_used = 0
        for j in range(m):
            Z[:, j] = M(V[:, j])
            w = matvec(Z[:, j])
            # CGS2: two classical Gram-Schmidt passes
            Vh = V[:, :j + 1].conj().T if cplx else V[:, :j + 1].T
            h = Vh @ w
            w = w - V[:, :j + 1] @ h
            h2 = Vh @ w
            w = w - V[:, :j + 1] @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            Hm[:j + 1, j] = h
            Hm[j + 1, j] = hn
            if hn > 0.0:
                V[:, j + 1] = w / hn
            # apply the previous rotations, then make a new one
            # G_i = [[conj(c_i), s_i], [-s_i, c_i]] with s_i real (for real
            # input conj(c_i) = c_i: the real rotation)
            for i in range(j):
                ci = np.conj(cs[i]) if cplx else cs[i]
                t = ci * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            a, c = Hm[j, j], Hm[j + 1, j].real if cplx else Hm[j + 1, j]
            rho = np.sqrt(abs(a) ** 2 + c * c) if cplx else np.hypot(a, c)
            if rho == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j], sn[j] = a / rho, c / rho
            Hm[j, j] = rho
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = (np.conj(cs[j]) if cplx else cs[j]) * g[j]
            iters += 1
            j_used = j + 1
            if abs(g[j + 1]) <= tol * bnorm or hn == 0.0 or iters >= maxit:
                break
        # back substitution on the rotated (upper triangular) Hessenberg matrix
        y = np.zeros(j_used, dt)
        for i in range(j_used - 1, -1, -1):
            y[i] = (g[i] - Hm[i, i + 1:j_used] @ y[i + 1:]) / Hm[i, i]
        x = x + Z[:, :j_used] @ y
        restarts += 1


def richardson(matvec, b, precond, tol=1e-8, maxit=100):
    """Algorithm 1 step III: r = b - A x, err = ||r||/||b||, x <- x + M^-1 r,
    break when err < tol; then step IV error = ||A x - b||_2.  Real or
    complex (the complex kappa of Sec. 2): only sums, products and 2-norms."""
    b = np.asarray(b, dtype=np.result_type(b, np.float64))
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    errs = []
    it = 0
    for it in range(1, maxit + 1):
        r = b - matvec(x)
        err = np.linalg.norm(r) / bnorm
        errs.append(err)
        x = x + precond(r)
        if err < tol:
            break
    error = np.linalg.norm(matvec(x) - b)
    return x, {"iters": it, "history": errs, "error": error}

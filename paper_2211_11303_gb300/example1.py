"""Example 1 of the paper (Sec. 4): the unit cube with the constant current
J_S = [0, 0, 1]^T, beta = 1, H-LU preconditioned GMRES restarted after 100
steps and stopped at a relative residual of TOL = 1e-5, over the mesh levels
and wave numbers of Table 1.

The paper's coarse mesh of 6 tetrahedra refined k times is the Kuhn cube with
n = 2^(k-1) sub-cubes per side; its kappa (the coefficient of the mass term)
is kappa^2 here, so Table 1's 25 ... 900 are kappa = 5 ... 30.  The paper
computed in MATLAB; its iteration counts (TABLE1, as printed) are context for
the counts measured here, not a target: its H-matrix truncation parameters,
mesh generator and GMRES variant are not stated.

Run:  python -m paper_2211_11303_gb300.example1 [--n 2 4 8 16 32]
Every step runs in the library's kernels; this module only drives them.
"""
import argparse
import json
import time

# Table 1 (Sec. 4, Example 1): GMRES iteration counts by refinement level k
# and the paper's kappa (mass coefficient); None marks ">3000".
TABLE1_KAPPA = (25, 100, 225, 400, 625, 900)
TABLE1 = {
    2: (1, 1, 1, 1, 1, 1),
    3: (2, 2, 2, 2, 2, 2),
    4: (2, 4, 5, 5, 4, 3),
    5: (3, 4, 8, 9, 11, None),
    6: (3, 6, 20, 4, 48, 25),
    7: (4, 5, 7, 19, 46, 93),
}
J_S = (0.0, 0.0, 1.0)
TOL = 1e-5
RESTART = 100


def level_of(n):
    """Refinement level k of the Kuhn cube with n = 2^(k-1) sub-cubes per side."""
    k = n.bit_length()
    return k if n == 1 << (k - 1) else None


def run(ns=(2, 4, 8, 16, 32), kappas=(5, 10, 15, 20, 25, 30), leaf=32, eta=2.0, eps=1e-4, precision=None,
        maxit=3000):
    """One row per (n, kappa): iterations of FGMRES(100) to TOL 1e-5 on the
    constant-current load vector, with the paper's count beside it."""
    import torch

    from . import hlu

    prec = hlu.HLU_FP32 if precision is None else precision
    rows = []
    for n in ns:
        for kappa in kappas:
            t0 = time.perf_counter()
            h = hlu.hlu_build(n, float(kappa), leaf, eta, eps)
            try:
                hlu.hlu_factor(h, prec)
                info = hlu.hlu_factor_stats(h)
                N = hlu.hlu_n(h)
                b = torch.empty(N, dtype=torch.float64, device="cuda")
                hlu.hlu_rhs_constant_current(h, J_S, b)
                x = torch.empty_like(b)
                st = hlu.gmres_solve(h, b, x, restart=RESTART, tol=TOL, maxit=maxit, raise_on_nonconvergence=False)
                torch.cuda.synchronize()
            finally:
                hlu.hlu_destroy(h)
            k = level_of(n)
            col = TABLE1_KAPPA.index(kappa * kappa) if kappa * kappa in TABLE1_KAPPA else None
            paper = TABLE1[k][col] if (k in TABLE1 and col is not None) else None
            rows.append({"n": n, "k": k, "N": N, "kappa": kappa, "paper_kappa": kappa * kappa,
                         "iterations": st["iterations"], "converged": bool(st["converged"]),
                         "relres": st["relres_max"], "paper_iterations": paper,
                         "factor_ms": info["factor_ms"], "rank_max": info["rank_max"],
                         "rank_cap_hits": info["rank_cap_hits"], "wall_s": time.perf_counter() - t0})
    return rows


def main():
    ap = argparse.ArgumentParser(description="Example 1 (Sec. 4, Table 1) on the GPU")
    ap.add_argument("--n", type=int, nargs="+", default=[2, 4, 8, 16, 32])
    ap.add_argument("--kappa", type=float, nargs="+", default=[5, 10, 15, 20, 25, 30])
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--leaf", type=int, default=32)
    args = ap.parse_args()
    for r in run(args.n, [int(k) if float(k).is_integer() else k for k in args.kappa], leaf=args.leaf,
                 eps=args.eps):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()

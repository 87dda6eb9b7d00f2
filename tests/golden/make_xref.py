"""Writes the reference solutions of the n = 24 benchmark workload.

Test infrastructure: calls only the CPU oracle (oracle/, plain FP64) and
SciPy's sparse direct solver, never the GPU path.  For the Kuhn cube with
n = 24 sub-cubes per side (N = 91,656 interior edges) and kappa = 8 it
assembles A = K - kappa^2 M (Sec. 2.1 weak form), draws the 8 seeded N(0,1)
right-hand sides of the benchmark (synth.rhs_seed(2, 0, j), j = 0..7), and
solves A x = b by a sparse LU (SuperLU, COLAMD ordering) followed by one step
of iterative refinement in FP64.  The result is the x_ref of the forward error
||x - x_ref|| / ||x_ref|| that bench.py reports for the GPU solution (the
error the headline metric "solves/s to 1e-7 relative error" counts).

Output: xref_n24_kappa8.npy, float64 array of shape (N, 8), column j the
solution for right-hand side j, in the oracle's interior-edge DOF order (the
order of the library's vectors).  The relative residual of each column and the
size of the refinement correction are printed; both are below 1e-12, far
under the 1e-7 the metric checks.

Run from the repository root:  python tests/golden/make_xref.py
(about 4 minutes and 3 GB of host memory, single-threaded SuperLU).
"""
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import fem, mesh  # noqa: E402

N_CUBE, KAPPA, NRHS, CONFIG = 24, 8.0, 8, 2
OUT = os.path.join(HERE, "xref_n24_kappa8.npy")


def reference_solutions(n=N_CUBE, kappa=KAPPA, nrhs=NRHS, config=CONFIG):
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsc()
    N = A.shape[0]
    B = np.stack([synth.normal(synth.rhs_seed(config, 0, j), N) for j in range(nrhs)], axis=1)
    lu = spla.splu(A, permc_spec="COLAMD")
    X = lu.solve(B)
    R = A @ X - B
    X1 = X - lu.solve(R)
    relres = np.linalg.norm(A @ X1 - B, axis=0) / np.linalg.norm(B, axis=0)
    corr = np.linalg.norm(X1 - X, axis=0) / np.linalg.norm(X1, axis=0)
    return X1, relres, corr


if __name__ == "__main__":
    X, relres, corr = reference_solutions()
    print("relative residuals:", relres)
    print("refinement corrections:", corr)
    assert relres.max() < 1e-12 and corr.max() < 1e-10
    np.save(OUT, X)
    print("wrote", OUT, X.shape)

"""The stored reference solutions of the n = 24 benchmark workload
(tests/golden/xref_n24_kappa8.npy, written by tests/golden/make_xref.py from
the CPU oracle) solve the oracle's system: A x_ref = b for the benchmark's
seeded right-hand sides, to a relative residual far below the 1e-7 forward
error the metric counts.  No GPU."""
import os

import numpy as np

import synth
from oracle import fem, mesh

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stored_reference_solves_the_oracle_system():
    X = np.load(os.path.join(HERE, "golden", "xref_n24_kappa8.npy"))
    m = mesh.interior_edges(24)
    A = fem.assemble(m, 8.0).tocsr()
    N = A.shape[0]
    assert X.shape == (N, 8) and N == 91656
    B = np.stack([synth.normal(synth.rhs_seed(2, 0, j), N) for j in range(8)], axis=1)
    rel = np.linalg.norm(A @ X - B, axis=0) / np.linalg.norm(B, axis=0)
    assert rel.max() < 1e-12, rel

"""CPU FP64 oracle for H-LU preconditioned Nedelec edge-FEM solves of
time-harmonic Maxwell (Parvizi, Khodadadian, Beuchler, Wick: "Hierarchical LU
preconditioning for the time-harmonic Maxwell equations", arXiv 2211.11303).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the method (Sec. 2 weak form and Nedelec discretisation,
Sec. 3 H-matrices, Algorithm 1 I-IV, Sec. 4 cluster tree, admissibility,
truncated SVD, GMRES).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The GPU library (``paper_2211_11303_gb300``) never imports, links or calls it,
and it never imports the GPU library: the two share no code.  The only module
both sides use is ``synth`` (seeded random inputs, none of the method's
arithmetic).

Modules
  mesh     Kuhn-cube tetrahedral mesh, interior edges (Sec. 2.1)
  fem      element matrices, CSR assembly of A = K - kappa^2 M, RHS (Eq. 5-7)
  trees    geometric cluster tree and eta-admissible block tree (Sec. 3-4)
  hmatrix  A_H, truncation, recursive H-LU, H-triangular solves (Alg. 1 I, II)
  krylov   GMRES / flexible GMRES and the Richardson loop (Alg. 1 III-IV, Sec. 4)

Parity status of each function is stated in its module header.
"""

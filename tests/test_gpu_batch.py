"""Batched launches (through the C ABI): many problems' task DAGs in one
persistent launch must give exactly what one launch per problem gives (every
task computes the same thing whatever the interleaving), and the batch of
problems must meet the same parity bar as single problems."""
import numpy as np
import pytest

import synth

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


def _rhs(N, nrhs, seed):
    B = np.stack([synth.normal(seed + j, N) for j in range(nrhs)], axis=1)
    out = torch.empty((nrhs, N), dtype=torch.float64, device="cuda").t()  # column-major, ld = N
    out.copy_(torch.from_numpy(B))
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_factor_batch_equals_single(hlu, prec):
    P = hlu.HLU_FP32 if prec == "fp32" else hlu.HLU_FP64
    # batched workload recipe: mesh n and kappa drawn per problem (small sizes here)
    probs = [(4, 3.0), (5, 1.5), (6, 7.0), (5, 9.0), (3, 2.0)]
    single, batch = [], []
    try:
        for n, k in probs:
            single.append(hlu.hlu_build(n, k, 16, 2.0, 1e-4))
            batch.append(hlu.hlu_build(n, k, 16, 2.0, 1e-4))
        for h in single:
            hlu.hlu_factor(h, P)
        hlu.hlu_factor_batch(batch, P)
        for i, (hs, hb) in enumerate(zip(single, batch)):
            N = hlu.hlu_n(hs)
            b = _rhs(N, 2, 100 + i)
            x1 = hlu.colmajor(N, 2)
            x2 = hlu.colmajor(N, 2)
            hlu.hlu_solve(hs, b, x1)
            hlu.hlu_solve(hb, b, x2)
            torch.cuda.synchronize()
            assert torch.equal(x1, x2), i
            assert hlu.hlu_factor_stats(hb)["rank_max"] == hlu.hlu_factor_stats(hs)["rank_max"]
    finally:
        for h in single + batch:
            hlu.hlu_destroy(h)


def test_solve_batch_equals_single(hlu):
    probs = [(4, 2.0, 1), (6, 5.0, 3), (5, 1.0, 16), (6, 8.0, 7)]
    hs = []
    try:
        for n, k, _ in probs:
            h = hlu.hlu_build(n, k, 32, 2.0, 1e-4)
            hlu.hlu_factor(h, hlu.HLU_FP32)
            hs.append(h)
        bs, xs, refs = [], [], []
        for i, (h, (n, k, nr)) in enumerate(zip(hs, probs)):
            N = hlu.hlu_n(h)
            b = _rhs(N, nr, 200 + 16 * i)
            r = hlu.colmajor(N, nr)
            hlu.hlu_solve(h, b, r)
            bs.append(b)
            xs.append(hlu.colmajor(N, nr))
            refs.append(r)
        hlu.hlu_solve_batch(hs, bs, xs)
        torch.cuda.synchronize()
        for x, r in zip(xs, refs):
            assert torch.equal(x, r)
    finally:
        for h in hs:
            hlu.hlu_destroy(h)


def test_autotune_picks_a_measured_candidate(hlu):
    from paper_2211_11303_gb300 import autotune
    cands = [{"tile": 32, "compress_at": 48}, {"tile": 64, "compress_at": 32}]
    res = autotune.tune(5, 3.0, candidates=cands, nrhs=2)
    assert res["best"] in cands
    assert len(res["results"]) == 2 and all(r["converged"] for r in res["results"])
    assert res["best"]["tile"] == min(res["results"], key=lambda r: r["total_ms"])["tile"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_problems_meet_the_oracle_bars(hlu, prec):
    """Problems factored together in ONE batched launch, at the configuration
    of single-problem parity (leaf 32, eta 2), each meet the single-problem
    bars against the CPU oracle: the operator error ||z - (LU)_H^-1 A z|| /
    ||z|| within 2x of the oracle's recursive H-LU at equal eps, and the
    FGMRES solution within 1e-7 of the direct solve."""
    import scipy.sparse.linalg as spla

    from oracle import fem, hmatrix, mesh, trees

    P = hlu.HLU_FP32 if prec == "fp32" else hlu.HLU_FP64
    probs = [(6, 4.0, 1e-3), (8, 8.0, 1e-4), (10, 6.0, 1e-3)]
    hs = []
    try:
        for n, k, eps in probs:
            hs.append(hlu.hlu_build(n, k, 32, 2.0, eps))
        hlu.hlu_factor_batch(hs, P)
        for i, (h, (n, k, eps)) in enumerate(zip(hs, probs)):
            m = mesh.interior_edges(n)
            A = fem.assemble(m, k).tocsr()
            N = A.shape[0]
            perm, cl, bl = trees.build_trees(m, 32, 2.0)
            Z = np.stack([synth.normal(11 + j, N) for j in range(3)], axis=1)
            ref = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
            AZ = A @ Z
            e_or = max(np.linalg.norm(Z[:, j] - ref.apply(AZ[:, j])) / np.linalg.norm(Z[:, j]) for j in range(3))
            b = _rhs(N, 3, 0)
            b.copy_(torch.from_numpy(np.asfortranarray(AZ)))
            y = hlu.colmajor(N, 3)
            hlu.hlu_solve(h, b, y)
            torch.cuda.synchronize()
            Y = y.cpu().numpy()
            e_gpu = max(np.linalg.norm(Z[:, j] - Y[:, j]) / np.linalg.norm(Z[:, j]) for j in range(3))
            assert hlu.hlu_factor_stats(h)["rank_cap_hits"] == 0
            assert e_gpu <= 2.0 * e_or, (i, e_gpu, e_or)
            # GMRES on the batch-factored handle against the direct solve
            B = _rhs(N, 2, synth.rhs_seed(3, i, 0))
            x = hlu.colmajor(N, 2)
            st = hlu.gmres_solve(h, B, x, restart=50, tol=1e-10, maxit=500)
            torch.cuda.synchronize()
            xs = spla.splu(A.tocsc()).solve(B.cpu().numpy())
            xg = x.cpu().numpy()
            assert st["converged"] == 1
            for j in range(2):
                assert np.linalg.norm(xg[:, j] - xs[:, j]) <= 1e-7 * np.linalg.norm(xs[:, j]), (i, j)
    finally:
        for h in hs:
            hlu.hlu_destroy(h)

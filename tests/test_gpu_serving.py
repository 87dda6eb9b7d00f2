"""Continuous batching of GMRES solves through the C ABI: requests that join a
running batch, share factors and leave at different steps must each get the
result they get when solved alone (one request in the batch)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10          # GMRES tolerance of every request
MIX_VS_ALONE = 1e-9  # ||x_mix - x_alone|| / ||x_alone||


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


def _run(H, reqs, join_at):
    """reqs: (handle, b); request i joins at step join_at[i]; returns xs, stats."""
    xs = [H.colmajor(H.hlu_n(h), b.shape[1]) for h, b in reqs]
    states = [None] * len(reqs)
    done = [False] * len(reqs)
    stats = [None] * len(reqs)
    step = 0
    try:
        while not all(done):
            for i, (h, b) in enumerate(reqs):
                if states[i] is None and join_at[i] <= step:
                    states[i] = H.hlu_gmres_begin(h, b, xs[i], restart=50, tol=TOL, maxit=500)
            act = [g for i, g in enumerate(states) if g is not None and not done[i]]
            if act:
                H.hlu_gmres_step_batch(act)
            for i, g in enumerate(states):
                if g is not None and not done[i]:
                    d, st = H.hlu_gmres_status(g)
                    if d:
                        done[i] = True
                        stats[i] = st
            step += 1
            assert step < 2000
    finally:
        for g in states:
            if g is not None:
                H.hlu_gmres_end(g)
    torch.cuda.synchronize()
    return xs, stats


def test_mix_equals_alone(hlu):
    specs = [(4, 2.0), (5, 6.0), (6, 9.0)]
    hs = []
    try:
        for n, k in specs:
            h = hlu.hlu_build(n, k, 16, 2.0, 1e-4)
            hlu.hlu_factor(h, hlu.HLU_FP32)
            hs.append(h)
        # requests: (handle index, nrhs); two share handle 0 and two handle 2
        rq = [(0, 2), (1, 1), (0, 3), (2, 5), (2, 16), (1, 4)]
        reqs = [(hs[i], _rhs(hlu.hlu_n(hs[i]), nr, 7000 + 16 * j)) for j, (i, nr) in enumerate(rq)]
        mix, st_mix = _run(hlu, reqs, [0, 0, 1, 2, 2, 5])
        for j, (h, b) in enumerate(reqs):
            alone, st_alone = _run(hlu, [(h, b)], [0])
            assert st_mix[j]["converged"] and st_alone[0]["converged"]
            err = torch.linalg.norm(mix[j] - alone[0]) / torch.linalg.norm(alone[0])
            assert err <= MIX_VS_ALONE, (j, float(err))
            # and against the lockstep solver of a single request
            ref = hlu.colmajor(hlu.hlu_n(h), b.shape[1])
            hlu.gmres_solve(h, b, ref, restart=50, tol=TOL, maxit=500)
            err2 = torch.linalg.norm(mix[j] - ref) / torch.linalg.norm(ref)
            assert err2 <= MIX_VS_ALONE, (j, float(err2))
            # true residual of the served result
            r = hlu.colmajor(hlu.hlu_n(h), b.shape[1])
            hlu.hlu_spmv(h, mix[j], r)
            rel = torch.linalg.norm(r - b, dim=0) / torch.linalg.norm(b, dim=0)
            assert float(rel.max()) <= 10 * TOL
    finally:
        for h in hs:
            hlu.hlu_destroy(h)


def test_server_results_match_alone(hlu):
    """The request loop (admission by HBM budget, factor cache, one batched
    GMRES step for all running requests) returns for every request what a
    lone gmres_solve returns."""
    from paper_2211_11303_gb300 import serve
    import synth as S
    reqs = S.serving_requests(count=10, seed=5000, n_lo=3, n_hi=5, k_lo=1.0, k_hi=3.0, r_lo=1, r_hi=6, rate=50.0)
    for r in reqs:  # few distinct (n, kappa) keys so that the cache is used
        r["kappa"] = float(round(r["kappa"]))

    def rhs_of(req, N):
        return np.stack([S.normal(S.rhs_seed(4, req["id"], j), N) for j in range(req["nrhs"])], axis=1)

    # a budget that holds about two factors forces evictions
    probe = hlu.hlu_build(5, 1.0, 16, 2.0, 1e-4)
    fb = hlu.hlu_factor_bytes_estimate(probe, hlu.HLU_FP32)
    hlu.hlu_destroy(probe)
    srv = serve.Server(hbm_budget_bytes=3 * fb + 64 * serve.krylov_bytes(500, 16, 50), max_active=4, leaf=16,
                       restart=50, tol=TOL, maxit=500)
    try:
        res = srv.run(reqs, rhs_of)
    finally:
        srv.close()
    assert srv.stats["cache_hits"] > 0 and srv.stats["max_active"] > 1
    for r in res:
        h = hlu.hlu_build(r["n"], r["kappa"], 16, 2.0, 1e-4)
        try:
            hlu.hlu_factor(h, hlu.HLU_FP32)
            N = hlu.hlu_n(h)
            b = _rhs(N, r["nrhs"], 0)
            b.copy_(torch.from_numpy(rhs_of(r, N)))
            x = hlu.colmajor(N, r["nrhs"])
            hlu.gmres_solve(h, b, x, restart=50, tol=TOL, maxit=500)
            xs = torch.from_numpy(np.ascontiguousarray(r["x"])).cuda()
            err = torch.linalg.norm(xs - x) / torch.linalg.norm(x)
            assert r["converged"] and err <= MIX_VS_ALONE, (r["id"], float(err))
        finally:
            hlu.hlu_destroy(h)
        # and against the direct solve of the oracle's matrix (the metric's bar)
        from oracle import fem, mesh
        import scipy.sparse.linalg as spla
        A = fem.assemble(mesh.interior_edges(r["n"]), r["kappa"]).tocsc()
        xd = spla.splu(A).solve(rhs_of(r, A.shape[0]))
        xr = np.asarray(r["x"]).reshape(xd.shape)
        for j in range(xd.shape[1]):
            assert np.linalg.norm(xr[:, j] - xd[:, j]) <= 1e-7 * np.linalg.norm(xd[:, j]), (r["id"], j)
    summ = serve.latency_summary(res)
    assert summ["requests"] == len(reqs) and summ["p99_ms"] >= summ["p50_ms"] > 0


def test_result_unchanged_while_a_factorisation_runs(hlu):
    """A request's GMRES steps taken while another problem's factorisation
    runs on a second stream (hlu_factor_async, one CTA per SM) give the same
    result as the request alone, and the factorisation run beside them gives
    the same factor as one run alone."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    hs = hlu.hlu_build(5, 3.0, 16, 2.0, 1e-4)   # the running request's problem
    hb = hlu.hlu_build(16, 6.0, 32, 2.0, 1e-4)  # the problem factored beside it
    hb2 = hlu.hlu_build(16, 6.0, 32, 2.0, 1e-4)
    side = torch.cuda.Stream()
    try:
        hlu.hlu_factor(hs, hlu.HLU_FP32)
        hlu.hlu_factor(hb2, hlu.HLU_FP32)
        b = _rhs(hlu.hlu_n(hs), 3, 9100)
        alone, st_alone = _run(hlu, [(hs, b)], [0])
        # the same request, stepped while hb is factored on the side stream
        x = hlu.colmajor(hlu.hlu_n(hs), 3)
        with torch.cuda.stream(side):
            hlu.hlu_factor_async(hb, hlu.HLU_FP32, sms, side)
        g = hlu.hlu_gmres_begin(hs, b, x, restart=50, tol=TOL, maxit=500)
        steps_during = 0
        try:
            done = False
            while not done:
                hlu.hlu_gmres_step_batch([g])
                if not hlu.hlu_factor_wait(hb, block=False):
                    steps_during += 1
                done, st = hlu.hlu_gmres_status(g)
        finally:
            hlu.hlu_gmres_end(g)
        hlu.hlu_factor_wait(hb, block=True)
        torch.cuda.synchronize()
        assert steps_during > 0  # the steps did run while the factorisation was on the device
        err = torch.linalg.norm(x - alone[0]) / torch.linalg.norm(alone[0])
        assert st["converged"] and err <= MIX_VS_ALONE, float(err)
        # the factor computed beside the request equals one computed alone
        N = hlu.hlu_n(hb)
        z = _rhs(N, 2, 9200)
        y1, y2 = hlu.colmajor(N, 2), hlu.colmajor(N, 2)
        hlu.hlu_solve(hb, z, y1)
        hlu.hlu_solve(hb2, z, y2)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
    finally:
        for h in (hs, hb, hb2):
            hlu.hlu_destroy(h)

"""Autotuner of the factorisation granularity.

Two knobs shape the work of the H-LU task DAG without changing the method:
the dense tile size T (block-tree nodes whose row and column clusters both
hold at most T DOFs are factored as one exact dense tile, ``hlu_set_tile``)
and the stack width at which a truncation compresses (``hlu_set_trunc_params``).
The best pair depends on the mesh size and on the GPU; ``tune`` measures every
candidate on the problem it is given (build, factorisation and a preconditioned
FGMRES solve of seeded right-hand sides) and returns the fastest by the time
of one factorisation plus one solve of ``nrhs`` columns.  ``apply`` installs a
result for the hlu_build calls that follow.  Results are plain dicts and can be
stored with ``save`` / ``load`` (JSON) keyed by the workload; ``default_path``
names the store (the environment variable HLU_TUNED, else the one shipped
beside this module).
"""
import json
import os
import time

import numpy as np
import torch

from . import hlu as H

DEFAULT_CANDIDATES = [{"tile": t, "compress_at": c} for t in (32, 64) for c in (32, 48, 64, 80, 96)]


def default_path():
    """The result store: $HLU_TUNED when set and not empty, else tuned.json
    beside this module (the results measured for the shipped workloads)."""
    return os.environ.get("HLU_TUNED") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def apply(params):
    """Install a tuning result (or the defaults for None) process-wide."""
    params = params or {}
    H.hlu_set_tile(int(params.get("tile", 64)))
    H.hlu_set_trunc_params(int(params.get("compress_at", 0)), 0.0)


def _rhs(N, nrhs, seed):
    g = np.random.default_rng(seed)
    b = torch.empty((nrhs, N), dtype=torch.float64, device="cuda").t()
    b.copy_(torch.from_numpy(g.standard_normal((N, nrhs))))
    return b


def tune(n, kappa, leaf=32, eta=2.0, eps=1e-4, precision=H.HLU_FP32, nrhs=8, restart=50, tol=1e-10,
         candidates=None, seed=0):
    """Measure every candidate on the Kuhn n-cube problem; returns
    {"best": params, "results": [params + timings, ...]}."""
    results = []
    try:
        for cand in candidates or DEFAULT_CANDIDATES:
            apply(cand)
            h = H.hlu_build(n, kappa, leaf, eta, eps)
            try:
                N = H.hlu_n(h)
                H.hlu_factor(h, precision)  # first factorisation: allocation and warm-up
                t0 = time.perf_counter()
                H.hlu_factor(h, precision)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                b = _rhs(N, nrhs, seed)
                x = H.colmajor(N, nrhs)
                st = H.gmres_solve(h, b, x, restart=restart, tol=tol, maxit=10 * restart,
                                   raise_on_nonconvergence=False)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                results.append(dict(cand, factor_ms=1e3 * (t1 - t0), solve_ms=1e3 * (t2 - t1),
                                    total_ms=1e3 * (t2 - t0), iterations=st["iterations"],
                                    converged=bool(st["converged"])))
            finally:
                H.hlu_destroy(h)
    finally:
        apply(None)
    ok = [r for r in results if r["converged"]] or results
    best = min(ok, key=lambda r: r["total_ms"])
    return {"best": {"tile": best["tile"], "compress_at": best["compress_at"]}, "results": results,
            "workload": {"n": n, "kappa": kappa, "leaf": leaf, "eta": eta, "eps": eps, "nrhs": nrhs,
                         "precision": "fp32" if precision == H.HLU_FP32 else "fp64"}}


def save(path, result):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    w = result["workload"]
    data["n=%d,kappa=%g,eps=%g,%s" % (w["n"], w["kappa"], w["eps"], w["precision"])] = result
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load(path, n, kappa, eps, precision="fp32"):
    """The stored best parameters for a workload, or None."""
    try:
        with open(path) as f:
            data = json.load(f)
    except OSError:
        return None
    r = data.get("n=%d,kappa=%g,eps=%g,%s" % (n, kappa, eps, precision))
    return r["best"] if r else None

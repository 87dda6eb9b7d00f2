"""Critical-path analysis of one factorisation (or one triangular solve) from
the executor's per-task trace (``hlu_debug_factor_trace`` /
``hlu_debug_solve_trace``): per task kind the tasks and their summed run
time, the chain of latest-finishing predecessors that ends the launch (its
running time and the waits between its links), and the longest truncations
on it with their target sizes.

Run:  python -m paper_2211_11303_gb300.trace [--n 24] [--kappa 8] [--eps 1e-4]
Needs a GPU; the analysis of the returned trace runs on the host.
"""
import argparse
import ctypes
import json

import numpy as np

from . import hlu

TASK_BYTES = 136  # one task record (hlu_debug_task_record)


def _trace(h, solve=False, nrhs=8):
    L = hlu.lib()
    sizes = (ctypes.c_int64 * 2)()
    hp = ctypes.c_void_p(h)
    fn = L.hlu_debug_solve_trace if solve else L.hlu_debug_factor_trace
    arg = nrhs if solve else hlu.HLU_FP32
    hlu._check(fn(hp, arg, None, None, None, None, sizes))
    nt, ne = sizes[0], sizes[1]
    tr = np.zeros(4 * nt, np.uint64)
    pp = np.zeros(nt + 1, np.int64)
    pi = np.zeros(max(1, ne), np.int32)
    rec = np.zeros(TASK_BYTES * nt, np.uint8)
    hlu._check(fn(hp, arg, tr.ctypes.data_as(ctypes.c_void_p), pp.ctypes.data_as(ctypes.c_void_p),
                  pi.ctypes.data_as(ctypes.c_void_p), rec.ctypes.data_as(ctypes.c_void_p), sizes))
    tr = tr.reshape(nt, 4).astype(np.int64)
    tid = tr[:, 0] & ((1 << 40) - 1)
    start = np.zeros(nt, np.int64)
    end = np.zeros(nt, np.int64)
    claim = np.zeros(nt, np.int64)
    claim[tid], start[tid], end[tid] = tr[:, 1], tr[:, 2], tr[:, 3]
    t0 = claim.min()
    words = rec.reshape(nt, TASK_BYTES).view(np.int32).reshape(nt, TASK_BYTES // 4)
    return start - t0, end - t0, pp, pi, words


def analyse(h, solve=False, nrhs=8, top=20):
    """Summary dict of one traced launch on handle h (factorisation, or one
    solve of nrhs columns)."""
    s, e, pp, pi, words = _trace(h, solve, nrhs)
    typ = words[:, 0]
    pieces = words[:, 3]
    a_rows, b_rows = words[:, 8], words[:, 16]
    dur = e - s
    kinds = hlu.TASK_KINDS
    out = {"tasks": int(len(typ)), "span_ms": float(e.max() / 1e6), "kinds": {}, "path": {}}
    for k, name in enumerate(kinds):
        m = typ == k
        if m.any():
            out["kinds"][name] = {"tasks": int(m.sum()), "run_ms_sum": float(dur[m].sum() / 1e6),
                                  "mean_us": float(dur[m].mean() / 1e3)}
    i = int(np.argmax(e))
    path = []
    while True:
        path.append(i)
        p0, p1 = pp[i], pp[i + 1]
        if p1 == p0:
            break
        preds = pi[p0:p1]
        i = int(preds[np.argmax(e[preds])])
    path = np.array(path[::-1])
    out["path"]["tasks"] = int(len(path))
    out["path"]["run_ms"] = float(dur[path].sum() / 1e6)
    out["path"]["wait_ms"] = float((s[path[1:]] - e[path[:-1]]).sum() / 1e6) if len(path) > 1 else 0.0
    out["path"]["kinds"] = {}
    for k, name in enumerate(kinds):
        m = typ[path] == k
        if m.any():
            out["path"]["kinds"][name] = {"tasks": int(m.sum()), "run_ms": float(dur[path][m].sum() / 1e6)}
    tk = kinds.index("TRUNC")
    tp = path[typ[path] == tk]
    order = np.argsort(-dur[tp])[:top]
    out["path"]["longest_truncations"] = [
        {"us": float(dur[t] / 1e3), "rows": int(a_rows[t]), "cols": int(b_rows[t]), "pieces": int(pieces[t])}
        for t in tp[order]]
    return out


def main():
    ap = argparse.ArgumentParser(description="critical path of one factorisation / solve from the executor trace")
    ap.add_argument("--n", type=int, default=24)
    ap.add_argument("--kappa", type=float, default=8.0)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--leaf", type=int, default=32)
    ap.add_argument("--tuned", default=None, help="autotuner store to apply (tuned.json)")
    args = ap.parse_args()
    if args.tuned:
        from . import autotune
        best = autotune.load(args.tuned, args.n, args.kappa, args.eps, "fp32")
        if best:
            autotune.apply(best)
    hlu.hlu_set_wait_limit_ms(60000)
    h = hlu.hlu_build(args.n, args.kappa, args.leaf, 2.0, args.eps)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP32)
        info = hlu.hlu_factor_stats(h)
        res = {"factor_ms": info["factor_ms"], "factor": analyse(h), "solve": analyse(h, solve=True)}
    finally:
        hlu.hlu_destroy(h)
    print(json.dumps(res))


if __name__ == "__main__":
    main()

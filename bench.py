#!/usr/bin/env python
"""Benchmark of the H-LU preconditioned GMRES hot path on GB300.

Workload (default): Kuhn cube n = 24 (N = 91,656 interior edges), kappa = 8,
leaf 32, eta 2, eps 1e-4; FP32 H-LU factor, FP64 flexible GMRES(50) to a
relative residual of 1e-10; 8 seeded N(0,1) right-hand sides.

One step = the whole hot path on one batch: hlu_build (GPU mesh, assembly,
cluster tree, block tree, A_H descriptors; the task DAG is compiled once per
block-tree structure and reused), hlu_factor (FP32) and gmres_solve of the 8
right-hand sides.  `value` = solves per second with the right-hand sides
resident in HBM; `e2e` = the same with the right-hand sides copied from pinned
host memory and the solutions copied back inside the timed region.

Accuracy: after the timed region the solutions of the last step are compared
with the stored direct-solve reference of the same workload
(tests/golden/xref_n24_kappa8.npy, written by tests/golden/make_xref.py from
the CPU oracle's matrix); `accuracy.fwd_err_max` is the largest
||x - x_ref|| / ||x_ref|| over the right-hand sides, the error the metric's
"to 1e-7" counts.  `fp64_arm` times the plain FP64 factor + FP64 GMRES path on
the same workload, and `same_sample` times the GPU path on the CPU oracle's
own sample next to `cpu_baseline`.

`--impl reference` times the CPU oracle (oracle/, plain FP64 NumPy), as it
stands, on a bounded sample of the workload family.

Multi-GPU: the method does not shard (replicas only); with torchrun each rank
runs an independent replica, `value` sums the solves of all ranks over the
slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "H-LU-preconditioned GMRES solves/s to 1e-7 rel. error; factor GFLOP/s; p99 ms"
UNIT = "solves/s"


def _blob_sha1(path):
    """git's object id of a file's contents (what `git hash-object` prints)."""
    import hashlib
    with open(path, "rb") as f:
        data = f.read()
    return hashlib.sha1(b"blob %d\0" % len(data) + data).hexdigest()


def _factor_traffic(n, eps, precision, key="exec_kernel_factor", nrhs=None):
    """DRAM bytes per factorisation (key exec_kernel_factor) or preconditioner
    apply (exec_kernel_apply) launch recorded from an ncu capture in
    profiles/traffic.json, or None when that record is of another workload or
    the executor source changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[key]
        same_src = rec["exec_cu_blob"] == _blob_sha1(os.path.join(ROOT, "paper_2211_11303_gb300", "csrc", "exec.cu"))
        same_work = int(rec["n"]) == n and float(rec["eps"]) == eps and rec["precision"] == precision and (
            nrhs is None or int(rec.get("nrhs", -1)) == nrhs)
        return int(rec["dram_bytes_per_launch"]) if same_src and same_work else None
    except (OSError, KeyError, ValueError):
        return None


XREF = os.path.join(ROOT, "tests", "golden", "xref_n24_kappa8.npy")


def forward_errors(X, n, kappa, nrhs, rank):
    """Per right-hand side ||x - x_ref|| / ||x_ref|| against the stored direct
    solve of the n = 24, kappa = 8 workload (rank 0's seeds); None for another
    workload."""
    import numpy as np
    if n != 24 or kappa != 8.0 or rank != 0 or not os.path.exists(XREF):
        return None
    ref = np.load(XREF)
    if nrhs > ref.shape[1]:
        return None
    ref = ref[:, :nrhs]
    return (np.linalg.norm(X - ref, axis=0) / np.linalg.norm(ref, axis=0)).tolist()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(n=8, kappa=8.0, eps=1e-4, tol=1e-10):
    """One bounded oracle sample: the complete CPU path (assembly, trees, A_H,
    recursive H-LU, FGMRES) for one seeded N(0,1) right-hand side on the n-cube.
    Returns (seconds, iterations, N)."""
    import synth
    from oracle import fem, hmatrix, krylov, mesh, trees
    t0 = time.perf_counter()
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    perm, cl, bl = trees.build_trees(m, 32, 2.0)
    P = hmatrix.HLUPreconditioner(A, perm, cl, bl, eps)
    b = synth.normal(synth.rhs_seed(2, 0, 0), A.shape[0])
    x, info = krylov.fgmres(lambda v: A @ v, b, precond=P.apply, restart=50, tol=tol)
    return time.perf_counter() - t0, info["iters"], A.shape[0]


def cpu_baseline_subprocess(n=8):
    """Oracle sample in a single-threaded child process (BLAS threads = 1)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,bench;s,it,N=bench.oracle_sample(%d);print(json.dumps([s,it,N]))" % n)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    s, it, N = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / s, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": ("complete oracle path (assembly, trees, A_H, recursive FP64 H-LU, FGMRES to 1e-10) "
                       "for 1 seeded RHS on the n=%d cube (N=%d, kappa=8, eps 1e-4), single-threaded "
                       "(BLAS threads 1) on one of the host's %d cores: %.2f s, %d iterations; the oracle cannot "
                       "finish the n=24 factorisation within minutes" % (n, N, os.cpu_count(), s, it)),
            "seconds": s, "iterations": it}


def oracle_config(n):
    """Config of the CPU oracle's sample (what the reference arm and the
    cpu_baseline leg time)."""
    N = n_dofs(n)
    return {"workload": "Kuhn cube n=%d (N=%d), kappa=8, leaf 32, eta 2, eps 0.0001, FP64 H-LU + FP64 FGMRES(50) "
                        "to 1e-10, 1 seeded N(0,1) RHS (the oracle's bounded sample of the workload family)" % (n, N),
            "n": n, "N": N, "kappa": 8.0, "leaf": 32, "eta": 2.0, "eps": 1e-4, "nrhs": 1, "restart": 50,
            "tol": 1e-10, "precision": "fp64"}


def slowest_replica(dist, t_ms, e2e_ms, device):
    """Replicas only: every rank solves its own problem; the job takes as long
    as its slowest rank (max over ranks of both timings)."""
    if dist is None:
        return t_ms, e2e_ms
    import torch
    tt = torch.tensor([t_ms, e2e_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt[0]), float(tt[1])


def job_throughput(nrhs, steps, world, ms):
    """Solves per second of the whole job: every rank solves nrhs columns per step."""
    return nrhs * steps * world / (ms / 1000.0)


def n_dofs(n):
    """Interior edges of the Kuhn n-cube: 7n^3 - 9n^2 + 3n."""
    return 7 * n ** 3 - 9 * n ** 2 + 3 * n


def arm_config(args, world=1):
    n, N = args.n, n_dofs(args.n)
    return {"workload": "Kuhn cube n=%d (N=%d), kappa=%g, leaf %d, eta %g, eps %g, %s H-LU + FP64 "
                        "FGMRES(%d) to %g, %d seeded N(0,1) RHS" % (n, N, args.kappa, args.leaf, args.eta, args.eps,
                                                                   args.precision.upper(), args.restart, args.tol,
                                                                   args.nrhs),
            "n": n, "N": N, "kappa": args.kappa, "leaf": args.leaf, "eta": args.eta, "eps": args.eps,
            "tile": args.tile, "nrhs": args.nrhs, "restart": args.restart, "tol": args.tol,
            "parallelism": "replicas" if world > 1 else "single GPU"}


def serving_run(args):
    """Continuous-batching serving: Poisson arrivals of requests with mesh
    n ~ U{lo..hi}, kappa ~ U[1, 12], 1..16 seeded N(0,1) RHS each, served by
    paper_2211_11303_gb300.serve (factor cache, HBM-budget admission,
    factorisations on a side stream beside the running requests' GMRES
    steps).  Start-up first puts the task DAGs of the mesh catalogue in the
    library's schedule cache (host threads in parallel).  With --serve-c5 the
    arrival rate is 0.7x the capacity calibrated on a burst of requests from
    the same distribution; otherwise --serve-rate."""
    import concurrent.futures as cf

    import numpy as np

    import synth
    from paper_2211_11303_gb300 import hlu, serve

    lo, hi = args.serve_n_lo, args.serve_n_hi
    prec = hlu.HLU_FP32 if args.precision == "fp32" else hlu.HLU_FP64
    hlu.hlu_set_schedule_cache(64, 48 << 30)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        list(ex.map(lambda n: hlu.hlu_destroy(hlu.hlu_build(n, 1.0, args.leaf, args.eta, args.eps)),
                    range(hi, lo - 1, -1)))
    prewarm_s = time.perf_counter() - t0

    def rhs_of(req, N):
        return np.stack([synth.normal(synth.rhs_seed(4, req["id"], j), N) for j in range(req["nrhs"])], axis=1)

    def serve_once(reqs):
        srv = serve.Server(hbm_budget_bytes=args.serve_budget_gb * 1e9, max_active=64, leaf=args.leaf, eta=args.eta,
                           eps=args.eps, precision=prec, restart=args.restart, tol=args.tol, maxit=args.maxit)
        try:
            res = srv.run(reqs, rhs_of)
        finally:
            srv.close()
        return res, srv.stats

    rate = args.serve_rate
    calib = None
    if args.serve_c5:
        # capacity: a burst (every request at t = 0) of the same distribution
        burst = synth.serving_requests(count=args.serve_calib, seed=5100, n_lo=lo, n_hi=hi, k_lo=1.0, k_hi=12.0,
                                       r_lo=1, r_hi=16, rate=1e9)
        res_b, st_b = serve_once(burst)
        cap = len(burst) / st_b["wall_s"]
        rate = 0.7 * cap
        calib = {"requests": len(burst), "wall_s": st_b["wall_s"], "capacity_per_s": cap}
    reqs = synth.serving_requests(count=args.serving, seed=5000, n_lo=lo, n_hi=hi, k_lo=1.0, k_hi=12.0, r_lo=1,
                                  r_hi=16, rate=rate)
    res, stats = serve_once(reqs)
    summ = serve.latency_summary(res)
    out = dict(summ, rate_per_s=rate, n_range=[lo, hi], kappa_range=[1.0, 12.0], rhs_range=[1, 16],
               wall_s=stats["wall_s"], solves_per_s=summ["rhs_columns"] / stats["wall_s"],
               max_relres=max(r["relres"] for r in res), all_converged=all(r["converged"] for r in res),
               factorisations=stats["factorisations"], cache_hits=stats["cache_hits"],
               evictions=stats["evictions"], oom_retries=stats["oom_retries"], max_active=stats["max_active"],
               gmres_steps=stats["steps"],
               steps_during_factor=stats["steps_during_factor"], budget_gb=args.serve_budget_gb,
               schedule_prewarm_s=prewarm_s, overlap="factorisations on a side stream (1 CTA/SM) beside GMRES steps",
               note="latency = finish - arrival, including the request's own factorisation and any queueing")
    if calib:
        out["calibration"] = calib
        out["config"] = "C5: %d Poisson requests at 0.7x calibrated capacity" % args.serving
    return out


def batched_run(args):
    """Batched workload: `args.batched` seeded problems (mesh n ~ U{6..16},
    kappa ~ U[1, 10]) factored in ONE persistent launch, against one launch
    per problem."""
    import torch

    import synth
    from paper_2211_11303_gb300 import hlu

    prec = hlu.HLU_FP32 if args.precision == "fp32" else hlu.HLU_FP64
    probs = synth.batched_problems(count=args.batched, seed=3000, n_lo=6, n_hi=16, k_lo=1.0, k_hi=10.0)
    hs = [hlu.hlu_build(n, k, args.leaf, args.eta, args.eps) for n, k in probs]
    try:
        hlu.hlu_factor_batch(hs, prec)  # warm-up (allocation, first launch)
        torch.cuda.synchronize()
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            hlu.hlu_factor_batch(hs, prec)
        torch.cuda.synchronize()
        batched_ms = 1000.0 * (time.perf_counter() - t0) / reps
        t0 = time.perf_counter()
        for _ in range(reps):
            for h in hs:
                hlu.hlu_factor(h, prec)
        torch.cuda.synchronize()
        seq_ms = 1000.0 * (time.perf_counter() - t0) / reps
        flops = sum(hlu.hlu_factor_stats(h)["flops"] for h in hs)
        dofs = sum(hlu.hlu_n(h) for h in hs)
    finally:
        for h in hs:
            hlu.hlu_destroy(h)
    return {"problems": len(probs), "n_range": [6, 16], "kappa_range": [1.0, 10.0], "dofs_total": dofs,
            "batched_factor_ms": batched_ms, "one_launch_per_problem_ms": seq_ms,
            "speedup": seq_ms / batched_ms, "batched_factor_gflops": flops / (batched_ms / 1000.0) / 1e9}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample(args.ref_n)
    times = []
    for _ in range(args.steps):
        s, it, N = oracle_sample(args.ref_n)
        times.append(s)
    tot = sum(times)
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(oracle_config(args.ref_n), parallelism="single host core"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": ("each step: the complete FP64 oracle path (assembly, trees, A_H, recursive "
                                    "H-LU, FGMRES to 1e-10) for 1 seeded N(0,1) RHS on the n=%d cube (N=%d, "
                                    "kappa 8, eps 1e-4), a bounded stand-in for the workload; the oracle cannot "
                                    "factor the n=%d cube within minutes" % (args.ref_n, N, args.n))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def whole_path_run(hlu, n, kappa, leaf, eta, eps, prec, Bd, X, restart, tol, maxit, steps, warmup):
    """Times `steps` whole-path steps (hlu_build, hlu_factor, gmres_solve of
    Bd's columns into X) after `warmup` untimed ones; returns the mean step in
    ms and the last step's factor statistics and solve statistics."""
    import torch
    last = None
    times = []
    for k in range(warmup + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = hlu.hlu_build(n, kappa, leaf, eta, eps)
        try:
            hlu.hlu_factor(h, prec)
            info = hlu.hlu_factor_stats(h)
            st = hlu.gmres_solve(h, Bd, X, restart=restart, tol=tol, maxit=maxit)
        finally:
            hlu.hlu_destroy(h)
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(1000.0 * (time.perf_counter() - t0))
        last = (info, st)
    return statistics.mean(times), last[0], last[1]


def run_gpu(args):
    import numpy as np
    import torch

    import synth
    from paper_2211_11303_gb300 import _build, hlu

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _build.build()
    hlu.lib()
    hlu.hlu_set_wait_limit_ms(60000)
    # granularity: the autotuner's stored choice for this workload (or a fresh
    # tuning with --autotune), else the command-line tile
    from paper_2211_11303_gb300 import autotune
    tuned_path = autotune.default_path()
    prec_name = "fp32" if args.precision == "fp32" else "fp64"
    if args.autotune and rank == 0:
        res = autotune.tune(args.n, args.kappa, args.leaf, args.eta, args.eps,
                            hlu.HLU_FP32 if prec_name == "fp32" else hlu.HLU_FP64, nrhs=args.nrhs,
                            restart=args.restart, tol=args.tol)
        autotune.save(tuned_path, res)
    best = autotune.load(tuned_path, args.n, args.kappa, args.eps, prec_name)
    if best:
        autotune.apply(best)
        args.tile = int(best["tile"])
    else:
        hlu.hlu_set_tile(args.tile)
    n, kappa, nrhs = args.n, args.kappa, args.nrhs
    prec = hlu.HLU_FP32 if args.precision == "fp32" else hlu.HLU_FP64

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # inputs: seeded N(0,1) right-hand sides (config 2), resident on the device
    h0 = hlu.hlu_build(n, kappa, args.leaf, args.eta, args.eps)
    N = hlu.hlu_n(h0)
    hlu.hlu_destroy(h0)
    Bh = torch.empty((nrhs, N), dtype=torch.float64).pin_memory()
    for j in range(nrhs):
        Bh[j] = torch.from_numpy(synth.normal(synth.rhs_seed(2, rank, j), N))
    B = Bh.cuda().t()
    X = hlu.colmajor(N, nrhs)
    Xh = torch.empty((nrhs, N), dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()

    def step(copy_in=False, copy_out=False, rec=None):
        if copy_in:
            Bd = Bh.cuda(non_blocking=True).t()
        else:
            Bd = B
        h = hlu.hlu_build(n, kappa, args.leaf, args.eta, args.eps)
        try:
            hlu.hlu_factor(h, prec)
            info = hlu.hlu_factor_stats(h)
            g0 = time.perf_counter()
            st = hlu.gmres_solve(h, Bd, X, restart=args.restart, tol=args.tol, maxit=args.maxit)
            st["gmres_ms"] = 1000.0 * (time.perf_counter() - g0)
            if copy_out:
                Xh.copy_(X.t(), non_blocking=True)
        finally:
            hlu.hlu_destroy(h)
        if rec is not None:
            rec.append((info, st))

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    recs = []
    lat = []
    launches0 = hlu.hlu_launch_count()
    barrier()
    t_all0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        s0 = time.perf_counter()
        step(rec=recs)
        torch.cuda.synchronize()
        lat.append(1000.0 * (time.perf_counter() - s0))
    ev1.record(stream)
    barrier()
    dev_ms = ev0.elapsed_time(ev1)
    wall_ms = 1000.0 * (time.perf_counter() - t_all0)
    launches = hlu.hlu_launch_count() - launches0
    clk = clocks.stop()
    # end to end: host buffers in, host buffers out
    barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        step(copy_in=True, copy_out=True)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = 1000.0 * (time.perf_counter() - e0)

    # accuracy of the timed path: the last step's solutions (the e2e steps
    # rewrote X with the same solve) against the stored direct solve
    fwd = forward_errors(X.t().cpu().numpy().T, n, kappa, nrhs, rank)

    t_ms, e2e_ms = slowest_replica(dist, max(dev_ms, wall_ms), e2e_ms, "cuda")
    value = job_throughput(nrhs, args.steps, world, t_ms)
    e2e_value = job_throughput(nrhs, args.steps, world, e2e_ms)
    infos = [r[0] for r in recs]
    sts = [r[1] for r in recs]
    fl = statistics.mean(i["flops"] for i in infos)
    fms = statistics.mean(i["factor_ms"] for i in infos)
    peaks, src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 FMA pipe peak: 152 SMs x 128 lanes x 2 flop x max SM clock
    dev = torch.cuda.get_device_properties(local)
    fp32_peak_tflops = dev.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = fl / (fms / 1000.0) / 1e12
    lat_sorted = sorted(lat)
    p99 = lat_sorted[min(len(lat_sorted) - 1, int(round(0.99 * (len(lat_sorted) - 1))))]
    apply_ms = statistics.mean(s["precond_ms"] / max(s["precond_applies"], 1) for s in sts)
    live_bytes = statistics.mean(i["factor_live_bytes"] for i in infos)
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision.replace("fp", "f") + "+f64",
        "data": "synthetic",
        "config": dict(arm_config(args, world), l2="working set (factor %.2f GB) larger than L2"
                       % (infos[0]["factor_bytes"] / 1e9)),
        "factor_gflops": fl / (fms / 1000.0) / 1e9,
        "factor_ms": fms,
        "gmres_iterations": max(s["iterations"] for s in sts),
        "gmres_relres": max(s["relres_max"] for s in sts),
        "precond_ms_per_apply": apply_ms,
        "solve_phase": {"value": nrhs / (statistics.mean(s["gmres_ms"] for s in sts) / 1000.0), "unit": UNIT,
                        "note": "factor cached: the %d RHS columns of one step over the FGMRES time" % nrhs},
        "step_latency_ms": {"p50": statistics.median(lat), "p99": p99,
                            "note": "spread of the timed whole-path steps; the served p99 is p99_ms"},
        "schedule_ms_first_build": infos[0]["schedule_ms"],
        "rank_mean": statistics.mean(i["rank_mean"] for i in infos),
        "rank_max": max(i["rank_max"] for i in infos),
        "accuracy": {"fwd_err_max": max(fwd) if fwd else None, "fwd_err": fwd,
                     "target": 1e-7, "met": bool(fwd) and max(fwd) <= 1e-7,
                     "reference": ("stored direct solve of the oracle's matrix for these RHS "
                                   "(tests/golden/xref_n24_kappa8.npy: SuperLU + one refinement step, FP64)"
                                   if fwd else "no stored reference for this workload"),
                     "rank_cap_hits": max(i["rank_cap_hits"] for i in infos),
                     "rank_wanted_max": max(i["rank_wanted_max"] for i in infos),
                     "rank_capacity": 64},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak_tflops,
                     "traffic": _factor_traffic(n, args.eps, args.precision),
                     "kernel": "exec_kernel<float> (H-LU task executor), factorisation launch",
                     "peak_source": "derived: SMs x 128 FP32 lanes x 2 x %s max SM clock" % src,
                     "solve": {"bound": "hbm", "achieved": live_bytes / (apply_ms / 1000.0) / 1e9,
                               "peak": hbm_gbs, "unit": "GB/s",
                               "frac": live_bytes / (apply_ms / 1000.0) / 1e9 / hbm_gbs,
                               "traffic": _factor_traffic(n, args.eps, args.precision, "exec_kernel_apply", args.nrhs),
                               "bytes_per_apply": live_bytes,
                               "kernel": "exec_kernel<float> (H-LU task executor), one triangular-solve "
                                         "launch (L then U) per preconditioner apply",
                               "peak_source": "%s hbm_gbs" % src,
                               "note": "algorithmic bytes = factor words at their live ranks, read once per "
                                       "apply; time = CUDA events around the apply launches"}},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nrhs * N * 8,
                "d2h_bytes_per_step": nrhs * N * 8},
        "gpu_launches": launches,
        "autotune": best if best else "defaults (no stored tuning for this workload)",
    }
    if rank == 0 and args.fp64_steps > 0:
        # the plain FP64 path (FP64 factor and triangular solves, FP64 GMRES)
        # on the same workload and right-hand sides
        ms64, info64, st64 = whole_path_run(hlu, n, kappa, args.leaf, args.eta, args.eps, hlu.HLU_FP64, B, X,
                                            args.restart, args.tol, args.maxit, args.fp64_steps, 1)
        fwd64 = forward_errors(X.t().cpu().numpy().T, n, kappa, nrhs, rank)
        line["fp64_arm"] = {
            "value": nrhs / (ms64 / 1000.0), "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
            "factor_ms": info64["factor_ms"], "gmres_iterations": st64["iterations"],
            "precond_ms_per_apply": st64["precond_ms"] / max(st64["precond_applies"], 1),
            "fwd_err_max": max(fwd64) if fwd64 else None, "rank_cap_hits": info64["rank_cap_hits"],
            "ratio_fp32_over_fp64": value / world / (nrhs / (ms64 / 1000.0)),
            "note": "same workload, RHS and whole-path step (build + FP64 factor + FP64 GMRES), wall clock"}
    if rank == 0 and args.batched > 0:
        line["batched"] = batched_run(args)
    if rank == 0 and args.serving > 0:
        line["serving"] = serving_run(args)
        line["p99_ms"] = line["serving"]["p99_ms"]
        line["p50_ms"] = line["serving"]["p50_ms"]
    if rank == 0 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_subprocess(args.ref_n)
        except Exception as e:  # reported, not fatal
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                                    "kind": "oracle", "sample": "failed: %s" % e}
    if rank == 0 and args.same_sample_steps > 0:
        # the GPU whole path on the CPU oracle's own sample (n = ref_n, one
        # seeded RHS, kappa 8, eps 1e-4), in both factor precisions
        hs = hlu.hlu_build(args.ref_n, 8.0, 32, 2.0, 1e-4)
        Ns = hlu.hlu_n(hs)
        hlu.hlu_destroy(hs)
        bs = torch.from_numpy(synth.normal(synth.rhs_seed(2, 0, 0), Ns)).cuda().reshape(1, Ns).t()
        xs = hlu.colmajor(Ns, 1)
        same = {"config": oracle_config(args.ref_n), "steps": args.same_sample_steps}
        for name, pr in (("fp32_factor", hlu.HLU_FP32), ("fp64_factor", hlu.HLU_FP64)):
            ms_s, _, st_s = whole_path_run(hlu, args.ref_n, 8.0, 32, 2.0, 1e-4, pr, bs, xs, 50, 1e-10,
                                           args.maxit, args.same_sample_steps, 2)
            same[name] = {"value": 1000.0 / ms_s, "unit": UNIT, "ms_per_step": ms_s,
                          "gmres_iterations": st_s["iterations"]}
        cb = line.get("cpu_baseline", {}).get("value")
        if cb:
            same["gpu_over_oracle_fp32"] = same["fp32_factor"]["value"] / cb
            same["gpu_over_oracle_fp64"] = same["fp64_factor"]["value"] / cb
        line["same_sample"] = same
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=24)
    ap.add_argument("--kappa", type=float, default=8.0)
    ap.add_argument("--leaf", type=int, default=32)
    ap.add_argument("--eta", type=float, default=2.0)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--tile", type=int, default=64)
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--maxit", type=int, default=500)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--ref-n", type=int, default=8)
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the plain FP64 arm on the same workload (0: none)")
    ap.add_argument("--same-sample-steps", type=int, default=10,
                    help="timed GPU steps on the CPU oracle's sample (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="measure the tile / compression candidates on this workload first and store the best")
    ap.add_argument("--batched", type=int, default=64, help="problems of the batched-factor sample (0: none)")
    ap.add_argument("--serving", type=int, default=24, help="requests of the serving sample (0: none)")
    ap.add_argument("--serve-n-lo", type=int, default=8)
    ap.add_argument("--serve-n-hi", type=int, default=14)
    ap.add_argument("--serve-rate", type=float, default=4.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-c5", action="store_true",
                    help="serving at 0.7x the calibrated capacity (use with --serving 200 --serve-n-lo 8 "
                         "--serve-n-hi 32 for the full configuration)")
    ap.add_argument("--serve-calib", type=int, default=16, help="burst requests of the capacity calibration")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

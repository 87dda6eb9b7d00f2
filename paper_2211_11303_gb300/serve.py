"""Continuous-batching solve server on one GPU.

Each request asks for the solution of A(n, kappa) x = b for 1..16 right-hand
sides (Algorithm 1 steps III-IV of the paper: H-LU-preconditioned restarted
GMRES).  The server keeps H-LU factors on the device, keyed by (n, kappa), and
the Krylov state of every running request.  A request is admitted when a
slot is free and its factor (if not cached) plus its Krylov workspace fit the
HBM budget; cached factors that no running request uses are evicted, least
recently used first, to make room.  Every loop iteration advances ALL
running requests by one GMRES step through ``hlu_gmres_step_batch``: the
triangular solves of every request run in one persistent launch, and a
request's result is the same whether it ran alone or in the mix.

Arrivals follow the request's ``t`` (seconds after start) on the wall clock.
A request that needs a new factor is factored on a side stream
(``hlu_factor_async``) with the persistent launch capped at one CTA per SM,
while the loop keeps stepping the running requests on the main stream: the
executor holds two CTAs per SM, so the factorisation and the running
requests' triangular solves share every SM.  One factorisation is in flight
at a time; the request starts its GMRES once ``hlu_factor_wait`` reports the
factor done.  ``overlap=False`` factors synchronously in the loop instead
(the running requests wait for the factorisation).
"""
import time

import numpy as np
import torch

from . import hlu as H


def krylov_bytes(N, nrhs, restart):
    """Device bytes of one GMRES state (V, Z: N x (m+1) per column; W)."""
    return 8 * N * nrhs * (2 * (restart + 1) + 1) + 64 * 1024


class _Factor:
    def __init__(self, key, h, nbytes):
        self.key, self.h, self.nbytes = key, h, nbytes
        self.users = 0
        self.last_use = 0.0


def _device_room():
    """Device bytes a new allocation can get: the driver's free memory plus
    the whole segments PyTorch's caching allocator holds unused (free space
    inside partly used segments cannot serve a large block)."""
    st = torch.cuda.memory_stats()
    split = st.get("inactive_split_bytes.all.current", 0)
    return torch.cuda.mem_get_info()[0] + torch.cuda.memory_reserved() - torch.cuda.memory_allocated() - split


class Server:
    def __init__(self, hbm_budget_bytes, max_active=64, leaf=32, eta=2.0, eps=1e-4, precision=H.HLU_FP32,
                 restart=50, tol=1e-8, maxit=1000, overlap=True):
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.leaf, self.eta, self.eps = leaf, eta, eps
        self.precision, self.restart, self.tol, self.maxit = precision, restart, tol, maxit
        self.factors = {}
        self.used = 0
        self.reserve = 4 << 30  # device bytes kept free beyond each admission
        self.overlap = bool(overlap)
        self.side = torch.cuda.Stream() if self.overlap else None
        self.factor_ctas = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        self.inflight = None  # (entry of the request waiting for its factor, factor)
        self._active = []  # the running requests of run()
        self.stats = {"factorisations": 0, "cache_hits": 0, "evictions": 0, "steps": 0, "max_active": 0,
                      "steps_during_factor": 0, "oom_retries": 0}

    # -- factor cache ---------------------------------------------------------
    def _evict_for(self, need):
        idle = sorted((f for f in self.factors.values() if f.users == 0), key=lambda f: f.last_use)
        for f in idle:
            if self.used + need <= self.budget:
                break
            H.hlu_destroy(f.h)
            self.used -= f.nbytes
            del self.factors[f.key]
            self.stats["evictions"] += 1
        return self.used + need <= self.budget

    def _evict_one(self):
        """Free the least recently used cached factor no running request
        uses; False when there is none."""
        idle = sorted((f for f in self.factors.values() if f.users == 0), key=lambda f: f.last_use)
        if not idle:
            return False
        f = idle[0]
        H.hlu_destroy(f.h)
        self.used -= f.nbytes
        del self.factors[f.key]
        self.stats["evictions"] += 1
        torch.cuda.empty_cache()
        return True

    def _stuck(self, f=None):
        """Nothing runs or is being factored, and no cached factor but f
        exists: no memory will be released by waiting."""
        return not self._active and self.inflight is None and all(g is f for g in self.factors.values())

    def _room_for(self, need):
        """True once the device itself can hold `need` more bytes (beyond the
        reserve), evicting idle cached factors, least recently used first:
        schedules and handles live outside the budget, so the budget alone
        can admit what the device cannot hold."""
        while _device_room() <= need + self.reserve:
            if not self._evict_one():
                return False
        return True

    def _lookup(self, req, may_build=True):
        """(cached factor or None, built-but-unfactored handle or None, bytes);
        (None, None, 0) when the request needs a handle that may not be built
        now."""
        key = (int(req["n"]), float(req["kappa"]))
        f = self.factors.get(key)
        if f is not None:
            if "_h" in req:  # built while the factor was not cached yet
                H.hlu_destroy(req.pop("_h")[1])
            return f, None, 0
        if "_h" not in req:
            if not may_build:
                return None, None, 0
            h = None
            while h is None:
                try:
                    h = H.hlu_build(req["n"], req["kappa"], self.leaf, self.eta, self.eps)
                except H.HluError as e:
                    # the mesh's schedule or matrix did not fit: free an idle
                    # cached factor and build again, or wait for running
                    # requests to release memory
                    if e.status != "HLU_ERR_OOM":
                        raise
                    self.stats["oom_retries"] += 1
                    if self._evict_one():
                        continue
                    if self._stuck():
                        raise  # nothing held that could be released
                    return None, None, 0
            req["_h"] = (key, h, int(H.hlu_factor_bytes_estimate(h, self.precision)))
        return None, req["_h"], req["_h"][2]

    def prewarm(self, ns, kappa=1.0):
        """Build (and drop) one handle per mesh size so that the library's
        schedule cache holds the task DAGs of the mesh catalogue: a server
        start-up step, after which a request's latency holds its own
        factorisation and solve only."""
        for n in sorted(set(int(x) for x in ns)):
            H.hlu_destroy(H.hlu_build(n, kappa, self.leaf, self.eta, self.eps))

    @staticmethod
    def _columns(b):
        """Device right-hand sides (copied from the host array b, N x nrhs)
        and solution columns, each column contiguous."""
        N, nr = b.shape
        bd = torch.empty((nr, N), dtype=torch.float64, device="cuda").t()
        bd.copy_(torch.from_numpy(np.ascontiguousarray(b)).pin_memory(), non_blocking=True)
        xd = torch.empty((nr, N), dtype=torch.float64, device="cuda").t()
        return bd, xd

    def _start(self, req, f, N, kb, active):
        """Start the request's GMRES on factor f (admitted: f.users and kb
        already counted).  When the device cannot hold its columns or Krylov
        workspace, idle cached factors are freed, least recently used first,
        and the start retried; with none left the admission is undone and
        False returned, so the request waits for running ones to finish."""
        b = np.asarray(self._rhs_of(req, N), dtype=np.float64).reshape(N, -1)
        while True:
            try:
                bd, xd = self._columns(b)
                g = H.hlu_gmres_begin(f.h, bd, xd, restart=self.restart, tol=self.tol, maxit=self.maxit)
                break
            except (H.HluError, torch.cuda.OutOfMemoryError) as e:
                if isinstance(e, H.HluError) and e.status != "HLU_ERR_OOM":
                    raise
                bd = xd = None
                self.stats["oom_retries"] += 1
                if self._evict_one():
                    continue
                torch.cuda.empty_cache()
                f.users -= 1
                self.used -= kb
                if self._stuck(f):
                    raise  # nothing runs that could release memory
                return False
        active.append({"req": req, "f": f, "g": g, "b": bd, "x": xd, "kb": kb})
        return True

    # -- main loop --------------------------------------------------------------
    def run(self, requests, rhs_of):
        """Serve `requests` (dicts with id, t, n, kappa, nrhs) in arrival
        order; rhs_of(req, N) -> float64 host array (N, nrhs).  Returns one
        result dict per request (id, latency_s, iterations, relres, x)."""
        pending = sorted(requests, key=lambda r: (r["t"], r["id"]))
        self._rhs_of = rhs_of
        waiting, active, results = [], [], {}
        self._active = active
        t0 = time.perf_counter()
        pi = 0
        while pi < len(pending) or waiting or active or self.inflight is not None:
            now = time.perf_counter() - t0
            while pi < len(pending) and pending[pi]["t"] <= now:
                waiting.append(pending[pi])
                pi += 1
            # admission: first come first served, later requests may pass one
            # that does not fit yet
            # at most one request builds a new handle per pass: a handle holds
            # device memory (mesh, matrix, schedule state) before it is admitted
            still = []
            built_one = False
            for req in waiting:
                if len(active) + (self.inflight is not None) >= self.max_active:
                    still.append(req)
                    continue
                f, built, fbytes = self._lookup(req, may_build=not built_one)
                if f is None and built is not None and self.inflight is not None:
                    still.append(req)  # one factorisation in flight at a time
                    continue
                if f is not None and self.inflight is not None and f is self.inflight[1]:
                    still.append(req)  # its factor is being computed
                    continue
                if f is None and built is None:
                    still.append(req)
                    continue
                built_one = built_one or f is None
                N = H.hlu_n(f.h if f is not None else built[1])
                kb = krylov_bytes(N, req["nrhs"], self.restart)
                if f is not None:
                    f.users += 1  # not evictable while deciding
                ok = self._evict_for(fbytes + kb)
                # the device itself must have the room as well (schedules and
                # handles are outside the budget); blocks PyTorch's caching
                # allocator holds unused count as free
                ok = ok and self._room_for(fbytes + kb)
                if f is not None:
                    f.users -= 1
                if not ok:
                    if self._stuck(f):
                        raise RuntimeError("request %s needs %d bytes, more than the HBM budget or the device holds"
                                           % (req["id"], fbytes + kb))
                    if built is not None:  # do not hold an unadmitted handle's memory
                        H.hlu_destroy(req.pop("_h")[1])
                    still.append(req)
                    continue
                if f is None:
                    key, h, nbytes = req.pop("_h")
                    f = _Factor(key, h, nbytes)
                    self.factors[key] = f
                    self.used += nbytes + kb
                    self.stats["factorisations"] += 1
                    f.users += 1
                    try:
                        if self.overlap:
                            with torch.cuda.stream(self.side):
                                H.hlu_factor_async(h, self.precision, self.factor_ctas, self.side)
                            self.inflight = (req, f, N, kb)
                            continue
                        H.hlu_factor(h, self.precision)
                    except H.HluError as e:
                        # the device could not hold the factor after all
                        # (fragmented free memory): undo the admission and
                        # retry once running requests have released memory
                        if e.status != "HLU_ERR_OOM":
                            raise
                        del self.factors[key]
                        self.used -= nbytes + kb
                        self.stats["factorisations"] -= 1
                        self.stats["oom_retries"] += 1
                        H.hlu_destroy(h)
                        torch.cuda.empty_cache()
                        if self._stuck():
                            raise
                        still.append(req)
                        continue
                else:
                    self.stats["cache_hits"] += 1
                    f.users += 1
                    self.used += kb
                if not self._start(req, f, N, kb, active):
                    still.append(req)
            waiting = still
            if self.inflight is not None:
                # the factor of a newly admitted request: start its GMRES once
                # done (wait for it when nothing else can run meanwhile)
                req, f, N, kb = self.inflight
                if H.hlu_factor_wait(f.h, block=not active):
                    self.inflight = None
                    if not self._start(req, f, N, kb, active):
                        waiting.append(req)  # its factor stays cached
            if not active:
                if pi < len(pending) and self.inflight is None:
                    time.sleep(max(0.0, min(pending[pi]["t"] - (time.perf_counter() - t0), 0.05)))
                continue
            self.stats["max_active"] = max(self.stats["max_active"], len(active))
            H.hlu_gmres_step_batch([a["g"] for a in active])
            self.stats["steps"] += 1
            if self.inflight is not None:
                self.stats["steps_during_factor"] += 1
            keep = []
            for a in active:
                done, st = H.hlu_gmres_status(a["g"])
                if not done:
                    keep.append(a)
                    continue
                x = a["x"].t().contiguous().cpu().numpy().T
                t_done = time.perf_counter() - t0
                H.hlu_gmres_end(a["g"])
                a["f"].users -= 1
                a["f"].last_use = time.perf_counter()  # absolute: the order holds across run() calls
                self.used -= a["kb"]
                req = a["req"]
                results[req["id"]] = {"id": req["id"], "latency_s": t_done - req["t"], "iterations": st["iterations"],
                                      "relres": st["relres_max"], "converged": bool(st["converged"]), "x": x,
                                      "n": req["n"], "kappa": req["kappa"], "nrhs": req["nrhs"]}
            active[:] = keep  # the list _stuck reads
        self.stats["wall_s"] = time.perf_counter() - t0
        return [results[r["id"]] for r in requests]

    def close(self):
        if self.inflight is not None:
            H.hlu_factor_wait(self.inflight[1].h, block=True)
            self.inflight = None
        for f in self.factors.values():
            H.hlu_destroy(f.h)
        self.factors.clear()
        self.used = 0


def latency_summary(results):
    lat = np.array([r["latency_s"] for r in results]) * 1e3
    cols = sum(r["nrhs"] for r in results)
    return {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "rhs_columns": int(cols)}

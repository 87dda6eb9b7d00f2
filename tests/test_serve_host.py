"""Host logic of the continuous-batching server (admission, factor cache,
eviction, out-of-memory retries) against a fake of the library: a device
pool of fixed size from which handles, factors and Krylov workspaces are
taken, with the library's HLU_ERR_OOM when it runs out.  No GPU: the fake's
GMRES states finish after a fixed number of steps.  Covers the failure the
serving configuration met on the device: the Krylov workspace of a new
request failing to allocate ("alloc Z") while cached factors held the
memory it needed.
"""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2211_11303_gb300 import hlu as real_hlu  # noqa: E402
from paper_2211_11303_gb300 import serve  # noqa: E402

MB = 1 << 20


class FakeLib:
    """Device pool of `capacity` bytes; a handle of mesh n holds n MB, its
    factor 4 n MB, a GMRES state krylov_scale x the server's estimate."""

    HLU_FP32, HLU_FP64 = real_hlu.HLU_FP32, real_hlu.HLU_FP64
    HluError = real_hlu.HluError

    def __init__(self, capacity, krylov_scale=1.0, iters=3, build_fail=0):
        self.capacity, self.held = capacity, {}
        self.krylov_scale, self.iters = krylov_scale, iters
        self.next_id = 1
        self.calls = {"gmres_oom": 0, "build_oom": 0, "factor_oom": 0}
        self.build_fail = build_fail  # builds that fail first, whatever the room

    def free(self):
        return self.capacity - sum(self.held.values())

    def _take(self, key, nbytes, where):
        if nbytes > self.free():
            raise real_hlu.HluError("HLU_ERR_OOM", where + ": out of memory")
        self.held[key] = self.held.get(key, 0) + nbytes

    # handles
    def hlu_build(self, n, kappa, leaf, eta, eps):
        if self.build_fail:
            self.build_fail -= 1
            self.calls["build_oom"] += 1
            raise real_hlu.HluError("HLU_ERR_OOM", "upload factor schedule: out of memory")
        h = types.SimpleNamespace(id=self.next_id, n=int(n), factored=False, pending=0)
        self.next_id += 1
        self._take(("h", h.id), h.n * MB, "build")
        return h

    def hlu_destroy(self, h):
        assert ("h", h.id) in self.held, "destroyed twice"
        self.held.pop(("h", h.id))
        self.held.pop(("f", h.id), None)

    def hlu_n(self, h):
        return 100 * h.n

    def hlu_factor_bytes_estimate(self, h, precision):
        return 4 * h.n * MB

    def hlu_factor(self, h, precision):
        try:
            self._take(("f", h.id), 4 * h.n * MB, "alloc factor")
        except real_hlu.HluError:
            self.calls["factor_oom"] += 1
            raise
        h.factored = True

    def hlu_factor_async(self, h, precision, max_ctas, stream):
        self.hlu_factor(h, precision)
        h.pending = 2  # done at the second poll

    def hlu_factor_wait(self, h, block=False):
        h.pending = 0 if block else max(0, h.pending - 1)
        return h.pending == 0

    # GMRES states
    def hlu_gmres_begin(self, h, b, x, restart=50, tol=1e-8, maxit=1000):
        assert h.factored and ("h", h.id) in self.held
        N, nr = b.shape
        g = types.SimpleNamespace(id=self.next_id, steps=0, x=x, h=h)
        self.next_id += 1
        need = int(self.krylov_scale * serve.krylov_bytes(N, nr, restart))
        try:
            self._take(("g", g.id), need, "alloc Z")
        except real_hlu.HluError:
            self.calls["gmres_oom"] += 1
            raise
        return g

    def hlu_gmres_step_batch(self, states):
        for g in states:
            assert ("h", g.h.id) in self.held, "stepping a state whose factor was freed"
            g.steps += 1

    def hlu_gmres_status(self, g):
        done = g.steps >= self.iters
        if done:
            g.x.fill_(float(g.h.n))
        return done, {"iterations": g.steps, "relres_max": 1e-9, "converged": 1}

    def hlu_gmres_end(self, g):
        self.held.pop(("g", g.id))


@pytest.fixture
def fake(monkeypatch):
    def make(capacity, **kw):
        lib = FakeLib(capacity, **kw)
        monkeypatch.setattr(serve, "H", lib)
        monkeypatch.setattr(serve, "_device_room", lib.free)
        monkeypatch.setattr(serve.Server, "_columns", staticmethod(
            lambda b: (torch.from_numpy(np.ascontiguousarray(b.T)).t(), torch.zeros(b.shape[::-1], dtype=torch.float64).t())))
        monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
        monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
        monkeypatch.setattr(torch.cuda, "get_device_properties",
                            lambda d: types.SimpleNamespace(multi_processor_count=152))
        monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)

        class _Ctx:
            def __init__(self, s):
                pass

            def __enter__(self):
                return self

            def __exit__(self, *a):
                return False

        monkeypatch.setattr(torch.cuda, "stream", _Ctx)
        return lib
    return make


def _server(budget, overlap, **kw):
    srv = serve.Server(budget, max_active=kw.pop("max_active", 8), overlap=overlap, restart=4, **kw)
    srv.reserve = 0
    return srv


def _requests(ns, nrhs=2):
    return [{"id": i, "t": 0.0, "n": n, "kappa": 1.0, "nrhs": nrhs} for i, n in enumerate(ns)]


def _rhs(req, N):
    return np.full((N, req["nrhs"]), float(req["id"]))


def _check_results(reqs, res):
    assert [r["id"] for r in res] == [q["id"] for q in reqs]
    for q, r in zip(reqs, res):
        assert r["converged"] and r["iterations"] == 3
        assert r["x"].shape == (100 * q["n"], q["nrhs"]) and np.all(r["x"] == q["n"])


@pytest.mark.parametrize("overlap", [False, True])
def test_all_requests_served_and_memory_returned(fake, overlap):
    lib = fake(1 << 40)
    reqs = _requests([8, 8, 16, 8, 24, 16])
    srv = _server(1 << 40, overlap)
    res = srv.run(reqs, _rhs)
    _check_results(reqs, res)
    assert srv.stats["factorisations"] == 3 and srv.stats["cache_hits"] == 3
    assert srv.stats["oom_retries"] == 0
    assert srv.used == sum(f.nbytes for f in srv.factors.values())  # only cached factors remain counted
    srv.close()
    assert lib.free() == lib.capacity and srv.used == 0


@pytest.mark.parametrize("overlap", [False, True])
def test_gmres_start_out_of_memory_frees_idle_factors(fake, overlap):
    """The Krylov workspace is 6x the server's estimate, so admission passes
    but hlu_gmres_begin fails while idle cached factors hold the memory: the
    server frees them and starts the request (the failure of the serving
    run at budget 120 GB)."""
    # four handles and factors of n = 8 (40 MB each) and 4 MB: the fourth
    # request's admission sees 36 MB free (its factor and estimated workspace
    # need 33.2 MB), its factor leaves 4 MB, and its workspace takes 7.1 MB
    lib = fake(4 * 40 * MB + 4 * MB, krylov_scale=6.0)
    reqs = [{"id": i, "t": 0.0, "n": n, "kappa": 1.0 + i, "nrhs": 16} for i, n in enumerate([8, 8, 8, 8])]
    srv = _server(1 << 40, overlap, max_active=1)  # one at a time: earlier factors are idle when the next starts
    res = srv.run(reqs, _rhs)
    _check_results(reqs, res)
    assert lib.calls["gmres_oom"] >= 1 and srv.stats["oom_retries"] >= lib.calls["gmres_oom"]
    assert srv.stats["evictions"] >= 1
    srv.close()
    assert lib.free() == lib.capacity


def test_gmres_start_waits_for_running_requests(fake):
    """No idle factor to free: the request's admission is undone and it
    starts once a running request has released its workspace."""
    ws = int(6.0 * serve.krylov_bytes(800, 16, 4))  # 7.1 MB, six times the estimate
    # one factor (40 MB), two workspaces and 3 MB: the third request passes
    # admission (its estimate is 1.2 MB) and its workspace fails
    lib = fake(40 * MB + 2 * ws + 3 * MB, krylov_scale=6.0)
    reqs = [{"id": i, "t": 0.0, "n": 8, "kappa": 1.0, "nrhs": 16} for i in range(4)]
    srv = _server(1 << 40, False)
    res = srv.run(reqs, _rhs)
    _check_results(reqs, res)
    assert lib.calls["gmres_oom"] >= 1 and srv.stats["evictions"] == 0
    assert srv.stats["factorisations"] == 1
    srv.close()
    assert lib.free() == lib.capacity


def test_gmres_start_that_can_never_fit_raises(fake):
    lib = fake(40 * MB + 2 * serve.krylov_bytes(800, 16, 4), krylov_scale=50.0)  # admitted, never starts
    srv = _server(1 << 40, False)
    with pytest.raises(real_hlu.HluError, match="alloc Z"):
        srv.run(_requests([8], nrhs=16), _rhs)
    srv.close()
    assert lib.free() == lib.capacity


def test_build_out_of_memory_is_retried(fake):
    """hlu_build running out (the factor schedule's upload) with a cached
    idle factor: the factor is freed and the build repeated."""
    lib = fake(1 << 40)
    srv = _server(1 << 40, False)
    srv.run(_requests([8]), _rhs)
    lib.build_fail = 1
    reqs = _requests([16])
    res = srv.run(reqs, _rhs)
    _check_results(reqs, res)
    assert lib.calls["build_oom"] == 1 and srv.stats["evictions"] == 1
    srv.close()
    assert lib.free() == lib.capacity


def test_build_out_of_memory_with_nothing_held_raises(fake):
    lib = fake(1 << 40, build_fail=1)
    srv = _server(1 << 40, False)
    with pytest.raises(real_hlu.HluError, match="upload factor schedule"):
        srv.run(_requests([8]), _rhs)
    srv.close()
    assert lib.free() == lib.capacity


def test_budget_evicts_least_recently_used(fake):
    """The HBM budget holds two factors of n = 8 with their workspaces: a
    third mesh evicts the least recently used one."""
    lib = fake(1 << 40)
    kb = serve.krylov_bytes(800, 2, 4)
    srv = _server(2 * 32 * MB + kb, False, max_active=1)
    for kappa in (1.0, 2.0, 1.0, 3.0):
        srv.run([{"id": 0, "t": 0.0, "n": 8, "kappa": kappa, "nrhs": 2}], _rhs)
    assert set(srv.factors) == {(8, 1.0), (8, 3.0)}  # kappa 2 was the least recently used
    assert srv.stats["evictions"] == 1 and srv.stats["cache_hits"] == 1
    srv.close()
    assert lib.free() == lib.capacity


def test_request_above_budget_raises(fake):
    fake(1 << 40)
    srv = _server(10 * MB, False)
    with pytest.raises(RuntimeError, match="more than the HBM budget"):
        srv.run(_requests([8]), _rhs)
    srv.close()

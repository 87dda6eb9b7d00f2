"""Failure detection on the host side of the C ABI (no GPU fault is made):
an exact zero pivot in a diagonal leaf, a non-finite right-hand side, a
Krylov solve that runs out of iterations and a refused device allocation each
come back as a status, without a hang, and leave the device usable for the
next call."""
import time

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


def _solve_ok(hlu, n=5, kappa=3.0):
    """A normal build, factorisation and solve after a failure."""
    h = hlu.hlu_build(n, kappa, 16, 2.0, 1e-6)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64)
        N = hlu.hlu_n(h)
        b = torch.from_numpy(synth.normal(3, N)).cuda()
        x = torch.empty_like(b)
        st = hlu.gmres_solve(h, b, x, restart=30, tol=1e-10, maxit=100)
        assert st["converged"] == 1 and torch.isfinite(x).all()
    finally:
        hlu.hlu_destroy(h)


def test_zero_pivot_is_reported(hlu):
    h = hlu.hlu_build(4, 2.0, 16, 2.0, 1e-4)
    try:
        hlu.hlu_debug_zero_dof(h, 7)  # row and column 7 of A become zero
        with pytest.raises(hlu.HluError) as ei:
            hlu.hlu_factor(h, hlu.HLU_FP64)
        assert ei.value.status == "HLU_ERR_ZERO_PIVOT"
        with pytest.raises(hlu.HluError) as ei:
            hlu.hlu_factor(h, hlu.HLU_FP32)
        assert ei.value.status == "HLU_ERR_ZERO_PIVOT"
    finally:
        hlu.hlu_destroy(h)
    _solve_ok(hlu)


@pytest.mark.parametrize("solver", ["gmres", "richardson"])
def test_non_finite_rhs_is_rejected_at_once(hlu, solver):
    h = hlu.hlu_build(5, 3.0, 16, 2.0, 1e-6)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64)
        N = hlu.hlu_n(h)
        b = hlu.colmajor(N, 2)
        b.copy_(torch.from_numpy(np.stack([synth.normal(1, N), synth.normal(2, N)], axis=1)))
        b[17, 1] = float("nan")
        x = hlu.colmajor(N, 2)
        t0 = time.perf_counter()
        with pytest.raises(hlu.HluError) as ei:
            if solver == "gmres":
                hlu.gmres_solve(h, b, x, restart=30, tol=1e-10, maxit=1000)
            else:
                hlu.hlu_richardson(h, b, x, tol=1e-10, maxit=1000)
        assert ei.value.status == "HLU_ERR_ARG" and "not finite" in str(ei.value)
        assert time.perf_counter() - t0 < 5.0
        # the same handle solves a finite right-hand side afterwards
        b[17, 1] = 0.0
        st = hlu.gmres_solve(h, b, x, restart=30, tol=1e-10, maxit=100)
        assert st["converged"] == 1
    finally:
        hlu.hlu_destroy(h)


def test_maxit_exhaustion_writes_x_and_stats(hlu):
    h = hlu.hlu_build(6, 4.0, 32, 2.0, 1e-2)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP32)
        N = hlu.hlu_n(h)
        b = torch.from_numpy(synth.normal(9, N)).cuda()
        x = torch.full_like(b, float("nan"))
        with pytest.raises(hlu.HluError) as ei:
            hlu.gmres_solve(h, b, x, restart=30, tol=1e-14, maxit=2)
        assert ei.value.status == "HLU_ERR_NOT_CONVERGED"
        x.fill_(float("nan"))
        st = hlu.gmres_solve(h, b, x, restart=30, tol=1e-14, maxit=2, raise_on_nonconvergence=False)
        assert st["converged"] == 0 and st["iterations"] == 2 and st["precond_applies"] == 2
        assert torch.isfinite(x).all()  # the iterate after 2 steps, not the NaN fill
        assert 0.0 < st["relres_max"] < 1.0  # two steps reduce the residual from x = 0
    finally:
        hlu.hlu_destroy(h)
    _solve_ok(hlu)


def test_refused_allocation_is_oom_and_recoverable(hlu):
    # a first build puts this mesh's task DAG in the library's schedule cache
    # (device memory it keeps), so the handles below allocate only their own
    hlu.hlu_destroy(hlu.hlu_build(8, 2.0, 32, 2.0, 1e-4))
    base = hlu.hlu_device_bytes_in_use()
    try:
        hlu.hlu_set_device_memory_limit(base + (1 << 20))  # 1 MiB above what is held now
        with pytest.raises(hlu.HluError) as ei:
            hlu.hlu_build(8, 2.0, 32, 2.0, 1e-4)
        assert ei.value.status == "HLU_ERR_OOM"
        assert hlu.hlu_device_bytes_in_use() == base  # nothing leaked by the failed build
        hlu.hlu_set_device_memory_limit(0)
        h = hlu.hlu_build(8, 2.0, 32, 2.0, 1e-4)
        try:
            hlu.hlu_set_device_memory_limit(hlu.hlu_device_bytes_in_use() + (1 << 20))
            with pytest.raises(hlu.HluError) as ei:
                hlu.hlu_factor(h, hlu.HLU_FP32)  # the factor arena does not fit
            assert ei.value.status == "HLU_ERR_OOM"
            hlu.hlu_set_device_memory_limit(0)
            hlu.hlu_factor(h, hlu.HLU_FP32)  # the same handle factors once memory is there
        finally:
            hlu.hlu_destroy(h)
        assert hlu.hlu_device_bytes_in_use() == base
    finally:
        hlu.hlu_set_device_memory_limit(0)
    _solve_ok(hlu)


def test_gmres_start_out_of_memory_holds_nothing(hlu):
    """A GMRES state whose Krylov workspace cannot be had: HLU_ERR_OOM, and no
    device memory is held afterwards (the first workspace buffer, which fits,
    is freed again); the same call succeeds once the memory is there."""
    h = hlu.hlu_build(6, 3.0, 16, 2.0, 1e-4)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP64)
        N = hlu.hlu_n(h)
        nr, m = 2, 20
        b = hlu.colmajor(N, nr)
        b.copy_(torch.from_numpy(np.stack([synth.normal(11 + j, N) for j in range(nr)], axis=1)))
        x = hlu.colmajor(N, nr)

        def run_state():
            g = hlu.hlu_gmres_begin(h, b, x, restart=m, tol=1e-10, maxit=200)
            try:
                done, st = False, None
                for _ in range(400):
                    hlu.hlu_gmres_step_batch([g])
                    done, st = hlu.hlu_gmres_status(g)
                    if done:
                        break
                assert done and st["converged"] == 1, st
            finally:
                hlu.hlu_gmres_end(g)
            torch.cuda.synchronize()

        run_state()  # buffers the library creates on first use (solve terms, batch queue)
        base = hlu.hlu_device_bytes_in_use()
        first = 8 * N * (m + 1) * nr  # V, the first workspace buffer
        try:
            hlu.hlu_set_device_memory_limit(base + first + 4096)  # V fits, Z does not
            with pytest.raises(hlu.HluError) as ei:
                hlu.hlu_gmres_begin(h, b, x, restart=m, tol=1e-10, maxit=200)
            assert ei.value.status == "HLU_ERR_OOM"
            assert hlu.hlu_device_bytes_in_use() == base
        finally:
            hlu.hlu_set_device_memory_limit(0)
        run_state()  # the same start succeeds once the memory is there
        assert hlu.hlu_device_bytes_in_use() == base
    finally:
        hlu.hlu_destroy(h)
    _solve_ok(hlu)


def test_library_memory_comes_from_torch(hlu):
    """With the default binding the library's device memory comes from
    PyTorch's caching allocator (the allocator hook of the C ABI)."""
    torch.cuda.synchronize()
    before_t = torch.cuda.memory_allocated()
    before_l = hlu.hlu_device_bytes_in_use()
    h = hlu.hlu_build(8, 2.0, 32, 2.0, 1e-4)
    try:
        hlu.hlu_factor(h, hlu.HLU_FP32)
        held = hlu.hlu_device_bytes_in_use() - before_l
        assert held > 0
        assert torch.cuda.memory_allocated() - before_t >= held
    finally:
        hlu.hlu_destroy(h)
    assert hlu.hlu_device_bytes_in_use() == before_l

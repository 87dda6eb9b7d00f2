"""Thin ctypes binding of the C ABI in include/hlu.h.

Argument marshalling only: every numerical step runs in libhlu.so's CUDA
kernels.  PyTorch provides device memory and streams: on loading, the
library's device allocator is pointed at PyTorch's caching allocator
(hlu_set_allocator; set HLU_ALLOCATOR=cuda in the environment to keep
cudaMalloc).  Vectors are FP64 CUDA tensors of shape (N,) or (N, nrhs) in
column-major layout (``colmajor`` makes one), in the original interior-edge
DOF order.
"""
import ctypes
import os

from ._build import LIB

HLU_OK = 0
HLU_ERR_NOT_CONVERGED = 4
HLU_FP64 = 0
HLU_FP32 = 1
HLU_TF32 = 2
HLU_PRECOND_LU = 0
HLU_PRECOND_HINV = 1
HLU_HINV_MAX_ITERS = 64
BLOCK_ADM, BLOCK_DENSE, BLOCK_SUB = 0, 1, 2


class HluError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (status, message))
        self.status = status


class hlu_mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("nt", ctypes.c_int32), ("xyz", ctypes.c_void_p),
                ("tets", ctypes.c_void_p), ("lattice_n", ctypes.c_int32), ("beta", ctypes.c_void_p)]


class hlu_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("relres_max", ctypes.c_double), ("abs_res_max", ctypes.c_double),
                ("precond_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("precond_applies", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class hlu_factor_info(ctypes.Structure):
    _fields_ = [("n_tasks", ctypes.c_int64), ("n_solve_tasks", ctypes.c_int64),
                ("factor_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("flops", ctypes.c_double), ("factor_ms", ctypes.c_double),
                ("schedule_ms", ctypes.c_double), ("rank_max", ctypes.c_int32),
                ("rank_cap_hits", ctypes.c_int32), ("rank_mean", ctypes.c_double),
                ("n_clusters", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("n_adm", ctypes.c_int32), ("n_dense", ctypes.c_int32),
                ("rank_wanted_max", ctypes.c_int32), ("trunc_dense_fallbacks", ctypes.c_int32),
                ("factor_live_bytes", ctypes.c_int64), ("grid_ctas", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]


class hlu_hinv_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("n_residuals", ctypes.c_int32),
                ("residual", ctypes.c_double * (HLU_HINV_MAX_ITERS + 1)), ("alpha", ctypes.c_double),
                ("rank_max", ctypes.c_int32), ("reserved", ctypes.c_int32), ("rank_mean", ctypes.c_double),
                ("inverse_live_bytes", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("n_iter_tasks", ctypes.c_int64), ("schedule_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


def _struct_dict(s):
    return {f[0]: getattr(s, f[0]) for f in s._fields_}


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f64 = ctypes.c_double
_P = ctypes.POINTER

# exported symbol -> (restype, argtypes); kept in sync with include/hlu.h and
# include/hlu_debug.h (tests check every declared name is exported)
SIGNATURES = {
    "hlu_build": (_i32, [_P(hlu_mesh), _f64, _i32, _f64, _f64, _i32, _vp, _P(_vp)]),
    "hlu_mesh_kuhn_cube": (_i32, [_i32, _P(hlu_mesh)]),
    "hlu_mesh_free": (None, [_P(hlu_mesh)]),
    "hlu_n": (_i64, [_vp]),
    "hlu_set_schedule_cache": (_i32, [_i32, _i64]),
    "hlu_export_trees": (_i32, [_vp, _vp, _vp, _vp, _P(_i64)]),
    "hlu_export_csr": (_i32, [_vp, _vp, _vp, _vp, _P(_i64)]),
    "hlu_rhs_manufactured": (_i32, [_vp, _vp, _vp]),
    "hlu_rhs_manufactured_noalloc": (_i32, [_vp, _vp, _vp]),
    "hlu_rhs_constant_current": (_i32, [_vp, _f64, _f64, _f64, _vp, _vp]),
    "hlu_spmv": (_i32, [_vp, _vp, _vp, _i32, _i64, _vp]),
    "hlu_factor": (_i32, [_vp, _i32, _vp]),
    "hlu_factor_async": (_i32, [_vp, _i32, _i32, _vp]),
    "hlu_factor_wait": (_i32, [_vp, _i32, _P(_i32)]),
    "hlu_factor_stats": (_i32, [_vp, _P(hlu_factor_info)]),
    "hlu_factor_profile": (_i32, [_vp, _vp]),
    "hlu_solve": (_i32, [_vp, _vp, _vp, _i32, _i64, _vp]),
    "gmres_solve": (_i32, [_vp, _vp, _vp, _i32, _i64, _i32, _f64, _i32, _i32, _P(hlu_stats), _vp]),
    "hlu_richardson": (_i32, [_vp, _vp, _vp, _i32, _i64, _f64, _i32, _P(hlu_stats), _vp]),
    "hlu_factor_batch": (_i32, [_P(_vp), _i32, _i32, _vp]),
    "hlu_hinverse": (_i32, [_vp, _i32, _f64, _i32, _P(hlu_hinv_info), _vp]),
    "hlu_hinverse_apply": (_i32, [_vp, _vp, _vp, _i32, _i64, _vp]),
    "hlu_set_preconditioner": (_i32, [_vp, _i32]),
    "hlu_solve_batch": (_i32, [_P(_vp), _i32, _P(_vp), _P(_vp), _P(_i32), _vp]),
    "hlu_factor_bytes_estimate": (_i64, [_vp, _i32]),
    "hlu_set_wait_limit_ms": (None, [_f64]),
    "hlu_set_tile": (None, [_i32]),
    "hlu_set_trunc_params": (_i32, [_i32, _f64]),
    "hlu_launch_count": (_i64, []),
    "hlu_set_allocator": (_i32, [_vp, _vp, _vp]),
    "hlu_set_device_memory_limit": (_i32, [_i64]),
    "hlu_device_bytes_in_use": (_i64, []),
    "hlu_debug_zero_dof": (_i32, [_vp, _i64]),
    "hlu_debug_tf32_tile": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "hlu_gmres_begin": (_i32, [_vp, _vp, _vp, _i32, _i64, _i32, _f64, _i32, _vp, _P(_vp)]),
    "hlu_gmres_step_batch": (_i32, [_P(_vp), _i32, _vp]),
    "hlu_gmres_status": (_i32, [_vp, _P(_i32), _P(hlu_stats)]),
    "hlu_gmres_end": (None, [_vp]),
    "hlu_destroy": (None, [_vp]),
    "hlu_status_string": (ctypes.c_char_p, [_i32]),
    "hlu_last_error": (ctypes.c_char_p, []),
    "hlu_debug_host_factor_solve": (_i32, [_i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _f64, _i32,
                                           _i32, _i32, ctypes.c_uint64, _i32, _vp, _vp, _vp]),
    "hlu_debug_wait_timeout": (_i32, [_f64, _vp]),
    "hlu_debug_host_hinverse": (_i32, [_i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _f64, _i32, _i32, _f64, _i32,
                                       _i32, _vp, _vp, _vp]),
    "hlu_debug_host_factor_prefix": (_i32, [_i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _f64, _i32, _i32, _i32,
                                            ctypes.c_uint64, _i32, _vp, _vp, _vp, _i64, _vp, _vp]),
    "hlu_debug_factor_prefix": (_i32, [_vp, _i32, _i64, _vp, _vp, _vp]),
    "hlu_debug_task_record": (_i32, [_vp, _i64, _vp]),
    "hlu_debug_check_hazards": (_i32, [_i32, _vp, _i32, _vp, _i32, _i32, _i32, _i32, _i64, _vp]),
    "hlu_debug_factor_trace": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "hlu_debug_solve_trace": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "hlu_debug_truncate": (_i32, [_i32, _i32, _i32, _i32, _i32, _i32, _vp, _vp, ctypes.c_double, _i32, _vp, _vp, _vp,
                                  _vp]),
}


def lib():
    """Load libhlu.so; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libhlu.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        if os.environ.get("HLU_ALLOCATOR", "torch") != "cuda":
            use_torch_allocator()
    return _lib


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_torch_callbacks = None


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching
    allocator (on the current device and stream).  The callbacks are kept
    alive for the life of the process: the library may free blocks from
    handle finalisers late in interpreter shutdown, when they become no-ops."""
    global _torch_callbacks
    import atexit

    import torch

    if _torch_callbacks is None:
        state = {"down": False}

        def _alloc(nbytes, ctx, _t=torch, _s=state):
            try:
                return _t.cuda.caching_allocator_alloc(int(nbytes))
            except Exception:  # out of memory: the library reports HLU_ERR_OOM
                return None

        def _free(ptr, nbytes, ctx, _t=torch, _s=state):
            if _s["down"]:
                return
            try:
                _t.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        cbs = (_ALLOC_FN(_alloc), _FREE_FN(_free))
        for cb in cbs:  # never collected: the C side keeps the pointers
            ctypes.pythonapi.Py_IncRef(ctypes.py_object(cb))
        atexit.register(lambda s=state: s.__setitem__("down", True))
        _torch_callbacks = cbs
    _check(lib().hlu_set_allocator(ctypes.cast(_torch_callbacks[0], _vp), ctypes.cast(_torch_callbacks[1], _vp),
                                   None))


def use_cuda_allocator():
    """Back to cudaMalloc/cudaFree for allocations made from now on."""
    _check(lib().hlu_set_allocator(None, None, None))


def hlu_set_device_memory_limit(nbytes):
    _check(lib().hlu_set_device_memory_limit(int(nbytes)))


def hlu_device_bytes_in_use():
    return int(lib().hlu_device_bytes_in_use())


def hlu_debug_zero_dof(h, dof):
    _check(lib().hlu_debug_zero_dof(_vp(h), int(dof)))


def _check(status):
    if status not in (HLU_OK,):
        L = lib()
        raise HluError(L.hlu_status_string(status).decode(), L.hlu_last_error().decode())
    return status


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def colmajor(N, nrhs, device="cuda"):
    """Empty FP64 (N, nrhs) CUDA tensor with column-major strides (1, N)."""
    import torch
    return torch.empty((nrhs, N), dtype=torch.float64, device=device).t()


def _vec(t, N):
    """(pointer, nrhs, ld) of an FP64 CUDA vector/column-major block."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError("expected a float64 CUDA tensor")
    if t.dim() == 1:
        if t.stride(0) != 1 or t.shape[0] != N:
            raise ValueError("vector must be contiguous with N entries")
        return _vp(t.data_ptr()), 1, N
    if t.shape[0] != N or t.stride(0) != 1 or t.stride(1) < N:
        raise ValueError("expected column-major (N, nrhs) with stride (1, ld >= N)")
    return _vp(t.data_ptr()), t.shape[1], t.stride(1)


# ---------------------------------------------------------------- C-ABI names
def lattice_mesh(n, beta=None):
    """hlu_mesh of the Kuhn cube with n^3 sub-cubes (the lattice path); beta:
    optional float64 array of 6 n^3 material coefficients (kept alive by the
    caller while the struct is used)."""
    return hlu_mesh(0, 0, None, None, int(n), None if beta is None else beta.ctypes.data)


def hlu_mesh_kuhn_cube(n):
    """(xyz float64 [nv, 3], tets int32 [nt, 4]) of the library's Kuhn cube."""
    import numpy as np
    m = hlu_mesh()
    _check(lib().hlu_mesh_kuhn_cube(int(n), ctypes.byref(m)))
    try:
        xyz = np.ctypeslib.as_array(ctypes.cast(m.xyz, _P(ctypes.c_double)), shape=(m.nv, 3)).copy()
        tets = np.ctypeslib.as_array(ctypes.cast(m.tets, _P(ctypes.c_int32)), shape=(m.nt, 4)).copy()
    finally:
        lib().hlu_mesh_free(ctypes.byref(m))
    return xyz, tets


def _beta_array(beta, nt):
    import numpy as np
    if beta is None:
        return None
    b = np.ascontiguousarray(beta, dtype=np.float64).reshape(-1)
    if b.shape[0] != nt:
        raise ValueError("beta needs one value per tetrahedron (%d)" % nt)
    return b


def hlu_build_mesh(xyz, tets, kappa, leaf=32, eta=2.0, eps=1e-4, rank_cap=0, stream=None, beta=None):
    """Algorithm 1 step I for a general tetrahedral mesh: xyz (nv, 3) float64
    coordinates, tets (nt, 4) vertex ids (host arrays); beta: optional
    material coefficient per tetrahedron."""
    import numpy as np
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    b = _beta_array(beta, tets.shape[0])
    m = hlu_mesh(xyz.shape[0], tets.shape[0], xyz.ctypes.data, tets.ctypes.data, 0,
                 None if b is None else b.ctypes.data)
    h = _vp()
    _check(lib().hlu_build(ctypes.byref(m), float(kappa), int(leaf), float(eta), float(eps), int(rank_cap),
                           _stream(stream), ctypes.byref(h)))
    return h.value


def hlu_build(n, kappa, leaf=32, eta=2.0, eps=1e-4, rank_cap=0, stream=None, beta=None):
    """Algorithm 1 step I on the GPU for the Kuhn n-cube; returns an opaque
    handle (int).  beta: optional material coefficient per tetrahedron, in
    the order of hlu_mesh_kuhn_cube."""
    h = _vp()
    b = _beta_array(beta, 6 * int(n) ** 3)
    m = lattice_mesh(n, b)
    _check(lib().hlu_build(ctypes.byref(m), float(kappa), int(leaf), float(eta), float(eps),
                           int(rank_cap), _stream(stream), ctypes.byref(h)))
    return h.value


def hlu_set_schedule_cache(entries, nbytes):
    _check(lib().hlu_set_schedule_cache(int(entries), int(nbytes)))


def hlu_n(h):
    return int(lib().hlu_n(_vp(h)))


def hlu_destroy(h):
    lib().hlu_destroy(_vp(h))


def hlu_export_trees(h):
    """(perm int32[N], clusters int32[nc,12], blocks int32[nb,8]) as numpy arrays."""
    import numpy as np
    sizes = (_i64 * 2)()
    _check(lib().hlu_export_trees(_vp(h), None, None, None, sizes))
    N = hlu_n(h)
    perm = np.empty(N, dtype=np.int32)
    C = np.empty((sizes[0], 12), dtype=np.int32)
    B = np.empty((sizes[1], 8), dtype=np.int32)
    _check(lib().hlu_export_trees(_vp(h), perm.ctypes.data, C.ctypes.data, B.ctypes.data, sizes))
    return perm, C, B


def hlu_export_csr(h):
    """(rowptr int64, col int32, val float64) numpy arrays of A."""
    import numpy as np
    nnz = _i64()
    _check(lib().hlu_export_csr(_vp(h), None, None, None, ctypes.byref(nnz)))
    N = hlu_n(h)
    rp = np.empty(N + 1, dtype=np.int64)
    ci = np.empty(nnz.value, dtype=np.int32)
    va = np.empty(nnz.value, dtype=np.float64)
    _check(lib().hlu_export_csr(_vp(h), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, ctypes.byref(nnz)))
    return rp, ci, va


def hlu_rhs_manufactured(h, b, stream=None):
    p, nr, ld = _vec(b, hlu_n(h))
    _check(lib().hlu_rhs_manufactured(_vp(h), p, _stream(stream)))


def hlu_rhs_constant_current(h, J, b, stream=None):
    """Load vector of the constant current density J = (jx, jy, jz)."""
    pb, nr, _ = _vec(b, hlu_n(h))
    if nr != 1:
        raise ValueError("b must be one column")
    _check(lib().hlu_rhs_constant_current(_vp(h), float(J[0]), float(J[1]), float(J[2]), pb, _stream(stream)))


def hlu_rhs_manufactured_noalloc(h, b, stream=None):
    """hlu_rhs_manufactured without allocations (fixed scratch, meshes n <= 24)."""
    pb, nr, _ = _vec(b, hlu_n(h))
    if nr != 1:
        raise ValueError("b must be one column")
    _check(lib().hlu_rhs_manufactured_noalloc(_vp(h), pb, _stream(stream)))


def hlu_spmv(h, x, y, stream=None):
    N = hlu_n(h)
    px, nr, ldx = _vec(x, N)
    py, nr2, ldy = _vec(y, N)
    if nr != nr2 or ldx != ldy:
        raise ValueError("x and y must have the same shape and leading dimension")
    _check(lib().hlu_spmv(_vp(h), px, py, nr, ldx, _stream(stream)))


def hlu_factor(h, precision=HLU_FP32, stream=None):
    _check(lib().hlu_factor(_vp(h), int(precision), _stream(stream)))


def hlu_factor_async(h, precision=HLU_FP32, max_ctas=0, stream=None):
    """Queue the factorisation on `stream` (capped at max_ctas CTAs) and return."""
    _check(lib().hlu_factor_async(_vp(h), int(precision), int(max_ctas), _stream(stream)))


def hlu_factor_wait(h, block=False):
    """True once the factorisation queued by hlu_factor_async has finished."""
    done = _i32()
    _check(lib().hlu_factor_wait(_vp(h), int(bool(block)), ctypes.byref(done)))
    return bool(done.value)


def hlu_factor_stats(h):
    info = hlu_factor_info()
    _check(lib().hlu_factor_stats(_vp(h), ctypes.byref(info)))
    return _struct_dict(info)


TASK_KINDS = ["GETRF", "TRSM_L", "TRSM_UT", "TRSM_U", "PROJ", "ROWMV", "TRUNC", "DADD", "RSOLVE", "FENCE"]


def hlu_factor_profile(h):
    """{kind: (tasks, wait_cycles, run_cycles)} of the last factorisation."""
    k0 = 3 * len(TASK_KINDS)
    out = (ctypes.c_uint64 * (k0 + 8))()
    _check(lib().hlu_factor_profile(_vp(h), out))
    d = {k: (out[3 * i], out[3 * i + 1], out[3 * i + 2]) for i, k in enumerate(TASK_KINDS)}
    d["trunc_phases"] = {"stack_cycles": out[k0], "qr_cycles": out[k0 + 1], "core_cycles": out[k0 + 2], "jacobi_cycles": out[k0 + 3],
                         "select_apply_cycles": out[k0 + 4], "compressions": out[k0 + 5], "sweeps": out[k0 + 6],
                         "width_sum": out[k0 + 7]}
    return d


def hlu_solve(h, b, x, stream=None):
    N = hlu_n(h)
    pb, nr, ldb = _vec(b, N)
    px, nr2, ldx = _vec(x, N)
    if nr != nr2 or ldb != ldx:
        raise ValueError("b and x must have the same shape and leading dimension")
    _check(lib().hlu_solve(_vp(h), pb, px, nr, ldb, _stream(stream)))


def gmres_solve(h, b, x, restart=50, tol=1e-8, maxit=1000, flexible=True, stream=None,
                raise_on_nonconvergence=True):
    """Restarted flexible GMRES with the H-LU preconditioner; returns stats dict."""
    N = hlu_n(h)
    pb, nr, ldb = _vec(b, N)
    px, nr2, ldx = _vec(x, N)
    if nr != nr2 or ldb != ldx:
        raise ValueError("b and x must have the same shape and leading dimension")
    st = hlu_stats()
    rc = lib().gmres_solve(_vp(h), pb, px, nr, ldb, int(restart), float(tol), int(maxit),
                           int(bool(flexible)), ctypes.byref(st), _stream(stream))
    if rc != HLU_ERR_NOT_CONVERGED or raise_on_nonconvergence:
        _check(rc)
    return _struct_dict(st)


def hlu_richardson(h, b, x, tol=1e-8, maxit=100, stream=None, raise_on_nonconvergence=True):
    N = hlu_n(h)
    pb, nr, ldb = _vec(b, N)
    px, nr2, ldx = _vec(x, N)
    st = hlu_stats()
    rc = lib().hlu_richardson(_vp(h), pb, px, nr, ldb, float(tol), int(maxit), ctypes.byref(st),
                              _stream(stream))
    if rc != HLU_ERR_NOT_CONVERGED or raise_on_nonconvergence:
        _check(rc)
    return _struct_dict(st)


def hlu_gmres_begin(h, b, x, restart=50, tol=1e-8, maxit=1000, stream=None):
    """Start a GMRES state for continuous batching; returns an opaque state."""
    N = hlu_n(h)
    pb, nr, ldb = _vec(b, N)
    px, nr2, ldx = _vec(x, N)
    if nr != nr2 or ldb != ldx:
        raise ValueError("b and x must have the same shape and leading dimension")
    g = _vp()
    _check(lib().hlu_gmres_begin(_vp(h), pb, px, nr, ldb, int(restart), float(tol), int(maxit),
                                 _stream(stream), ctypes.byref(g)))
    return g.value


def hlu_gmres_step_batch(states, stream=None):
    arr = (_vp * len(states))(*[_vp(g) for g in states])
    _check(lib().hlu_gmres_step_batch(arr, len(states), _stream(stream)))


def hlu_gmres_status(g):
    """(done, stats dict); raises nothing for non-convergence (see stats)."""
    done = _i32()
    st = hlu_stats()
    lib().hlu_gmres_status(_vp(g), ctypes.byref(done), ctypes.byref(st))
    return bool(done.value), _struct_dict(st)


def hlu_gmres_end(g):
    lib().hlu_gmres_end(_vp(g))


def hlu_hinverse(h, precision=HLU_FP32, tol=1e-10, maxit=HLU_HINV_MAX_ITERS, stream=None,
                 raise_on_nonconvergence=True):
    """Schulz inverse B_H of A_H; returns the record (residuals as a list)."""
    info = hlu_hinv_info()
    rc = lib().hlu_hinverse(_vp(h), int(precision), float(tol), int(maxit), ctypes.byref(info), _stream(stream))
    if rc != HLU_ERR_NOT_CONVERGED or raise_on_nonconvergence:
        _check(rc)
    d = _struct_dict(info)
    d["residual"] = [info.residual[k] for k in range(info.n_residuals)]
    return d


def hlu_hinverse_apply(h, b, x, stream=None):
    N = hlu_n(h)
    pb, nr, ldb = _vec(b, N)
    px, nr2, ldx = _vec(x, N)
    if nr != nr2 or ldb != ldx:
        raise ValueError("b and x must have the same shape and leading dimension")
    _check(lib().hlu_hinverse_apply(_vp(h), pb, px, nr, ldb, _stream(stream)))


def hlu_set_preconditioner(h, which):
    _check(lib().hlu_set_preconditioner(_vp(h), int(which)))


def hlu_factor_batch(handles, precision=HLU_FP32, stream=None):
    arr = (_vp * len(handles))(*[_vp(h) for h in handles])
    _check(lib().hlu_factor_batch(arr, len(handles), int(precision), _stream(stream)))


def hlu_solve_batch(handles, bs, xs, stream=None):
    n = len(handles)
    hs = (_vp * n)(*[_vp(h) for h in handles])
    pb = (_vp * n)()
    px = (_vp * n)()
    nr = (_i32 * n)()
    for i, (h, b, x) in enumerate(zip(handles, bs, xs)):
        N = hlu_n(h)
        p1, r1, l1 = _vec(b, N)
        p2, r2, l2 = _vec(x, N)
        if l1 != N or l2 != N or r1 != r2:
            raise ValueError("batched vectors must be dense column-major (ld = N)")
        pb[i], px[i], nr[i] = p1, p2, r1
    _check(lib().hlu_solve_batch(hs, n, pb, px, nr, _stream(stream)))


def hlu_factor_bytes_estimate(h, precision=HLU_FP32):
    return int(lib().hlu_factor_bytes_estimate(_vp(h), int(precision)))


def hlu_set_wait_limit_ms(ms):
    lib().hlu_set_wait_limit_ms(float(ms))


def hlu_launch_count():
    return int(lib().hlu_launch_count())


def hlu_set_trunc_params(compress_at=0, jacobi_tol=0.0):
    _check(lib().hlu_set_trunc_params(int(compress_at), float(jacobi_tol)))


def hlu_set_tile(t):
    lib().hlu_set_tile(int(t))



class Problem:
    """Owns one handle: build on construction, destroy on close()."""

    def __init__(self, n, kappa, leaf=32, eta=2.0, eps=1e-4, rank_cap=0, stream=None):
        self.n, self.kappa, self.leaf, self.eta, self.eps = n, kappa, leaf, eta, eps
        self.h = hlu_build(n, kappa, leaf, eta, eps, rank_cap, stream)
        self.N = hlu_n(self.h)

    def factor(self, precision=HLU_FP32, stream=None):
        hlu_factor(self.h, precision, stream)
        return hlu_factor_stats(self.h)

    def close(self):
        if self.h:
            hlu_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_truncate(X, Y, eps, cap=64, precision=HLU_FP64, piece_cols=0, flags=0):
    """One device truncation of X Y^T (numpy FP64 arrays m x w, n x w):
    (Xo m x r, Yo n x r, status words); flags as hlu_debug_truncate."""
    import numpy as np
    X = np.asfortranarray(X, dtype=np.float64)
    Y = np.asfortranarray(Y, dtype=np.float64)
    m, w = X.shape
    n = Y.shape[0]
    Xo = np.zeros((m, cap), order="F")
    Yo = np.zeros((n, cap), order="F")
    r = ctypes.c_int32(0)
    st = (ctypes.c_int32 * 8)()
    _check(lib().hlu_debug_truncate(int(precision), m, n, w, int(piece_cols), int(flags), X.ctypes.data, Y.ctypes.data,
                                    float(eps), int(cap), Xo.ctypes.data, Yo.ctypes.data, ctypes.byref(r), st))
    return Xo[:, :r.value].copy(), Yo[:, :r.value].copy(), list(st)

"""The library's host-side code under AddressSanitizer and
UndefinedBehaviorSanitizer (no GPU): the task scheduler, the host reference
executor of its DAGs, the race check and the host Schulz inverse, built with
g++ -fsanitize=address,undefined into tests/host_sanitize_driver.cpp and run
on the oracle's trees and matrix.  Any invalid access, leak or undefined
operation ends the run with an error; the solutions must equal those of the
normal library build."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import fem, mesh, trees

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2211_11303_gb300", "csrc")
SOURCES = [os.path.join(HERE, "host_sanitize_driver.cpp")] + [
    os.path.join(CSRC, s) for s in ("sched.cpp", "host_exec.cpp", "debug_api.cpp", "hazard.cpp")]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("hsan")
    exe = str(d / "host_sanitize_driver")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", *SOURCES, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "cannot find" in r.stderr:
        pytest.skip("sanitizer runtimes not installed")
    assert r.returncode == 0, r.stderr[-3000:]
    return exe, d


def _inputs(n, kappa, leaf, nrhs):
    m = mesh.interior_edges(n)
    A = fem.assemble(m, kappa).tocsr()
    perm, cl, bl = trees.build_trees(m, leaf, 2.0)
    p, C, B = trees.export_arrays(perm, cl, bl)
    N = A.shape[0]
    rng = np.random.default_rng(n)
    b = np.asfortranarray(rng.standard_normal((N, nrhs)))
    return A, p.astype(np.int32), C.astype(np.int32), B.astype(np.int32), b


def _library(A, p, C, B, b, tile, precision, seed):
    from paper_2211_11303_gb300 import hlu
    lib = hlu.lib()
    N, nrhs = b.shape
    x = np.zeros((N, nrhs), order="F")
    info = np.zeros(10, np.int64)
    rp = A.indptr.astype(np.int64)
    ci = A.indices.astype(np.int32)
    va = A.data.astype(np.float64)
    st = lib.hlu_debug_host_factor_solve(len(C), C.ctypes.data, len(B), B.ctypes.data, p.ctypes.data, rp.ctypes.data,
                                         ci.ctypes.data, va.ctypes.data, 1e-4, 32, tile, precision, seed, nrhs,
                                         b.ctypes.data, x.ctypes.data, info.ctypes.data)
    assert st == 0
    return x


@pytest.mark.parametrize("n,kappa,leaf,tile", [(3, 3.0, 16, 0), (4, 5.0, 16, 64)])
def test_host_code_is_clean_under_sanitizers(driver, n, kappa, leaf, tile):
    import __graft_entry__ as g
    g.build()
    exe, d = driver
    nrhs = 2
    A, p, C, B, b = _inputs(n, kappa, leaf, nrhs)
    N = A.shape[0]
    src, dst = str(d / ("in_%d.bin" % n)), str(d / ("out_%d.bin" % n))
    with open(src, "wb") as f:
        np.array([len(C), len(B), N, nrhs, tile], np.int32).tofile(f)
        np.array([A.nnz], np.int64).tofile(f)
        C.tofile(f)
        B.tofile(f)
        p.tofile(f)
        A.indptr.astype(np.int64).tofile(f)
        A.indices.astype(np.int32).tofile(f)
        A.data.astype(np.float64).tofile(f)
        np.ascontiguousarray(b.T).tofile(f)  # column-major: column by column
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([exe, src, dst], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-4000:])
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-4000:]
    out = np.fromfile(dst, np.float64).reshape(4, nrhs, N)
    xs = [o.T for o in out]
    # the sanitized build computes what the library computes
    for k, (prec, seed) in enumerate([(0, 0), (0, 3), (1, 0)]):
        xl = _library(A, p, C, B, b, tile, prec, seed)
        tol = 1e-12 if prec == 0 else 1e-5
        assert np.linalg.norm(xs[k] - xl) <= tol * np.linalg.norm(xl), (prec, seed)
    # any topological order gives the same result
    assert np.array_equal(xs[0], xs[1])
    # and both solve the system to the preconditioner's accuracy
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(xs[0] - xd) <= 1e-2 * np.linalg.norm(xd)
    assert np.all(np.isfinite(xs[3]))

"""Static race check of the task DAGs (hlu_debug_check_hazards, no GPU).

Every DAG the library launches (the H-LU factorisation of Algorithm 1 step II,
the triangular solve of step III, the Schulz inverse's start, step and apply)
is replayed over the element footprints of its tasks; every conflicting pair
of accesses must be ordered by the DAG's edges, and every access must stay in
its address space.  The check is itself tested by planted mistakes: removing
one edge must be reported unless another path still orders the two tasks.
"""
import numpy as np
import pytest

import synth
from oracle import mesh, trees

FACTOR, SOLVE, SCHULZ_START, SCHULZ_STEP, SCHULZ_APPLY = range(5)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2211_11303_gb300 import hlu
    return hlu.lib()


def _trees(n, leaf, general=False):
    if general:
        coords, tets = synth.perturbed_kuhn_mesh(n, 0.15, 7)
        m = mesh.general_mesh(coords, tets)
    else:
        m = mesh.interior_edges(n)
    perm, cl, bl = trees.build_trees(m, leaf, 2.0)
    return trees.export_arrays(perm, cl, bl)


def _check(lib, T, which, rank_cap=32, tile=0, nrhs=16, drop=-1):
    p, C, B = T
    rep = np.zeros(11, np.int64)
    st = lib.hlu_debug_check_hazards(len(C), C.ctypes.data, len(B), B.ctypes.data, rank_cap, tile, nrhs, which,
                                     drop, rep.ctypes.data)
    return st, rep


CONFIGS = [
    # (n, leaf, tile, rank capacity, general mesh)
    (4, 16, 0, 32, False),
    (4, 8, 16, 32, False),
    (5, 16, 32, 64, False),
    (6, 16, 64, 64, False),
    (5, 16, 32, 32, True),
    (3, 8, 0, 32, False),
    (4, 16, 32, 32, False),
]


@pytest.mark.parametrize("n,leaf,tile,cap,general", CONFIGS)
@pytest.mark.parametrize("which", [FACTOR, SOLVE, SCHULZ_START, SCHULZ_STEP, SCHULZ_APPLY])
def test_dag_orders_every_conflict(lib, n, leaf, tile, cap, general, which):
    st, rep = _check(lib, _trees(n, leaf, general), which, rank_cap=cap, tile=tile)
    if st == 6 and which == SCHULZ_STEP:
        pytest.skip("Schulz step DAG above the checker's 40,000 tasks")
    assert st == 0, rep
    assert rep[3] == 0 and rep[8] == 0, rep
    assert rep[0] > 0 and rep[1] > 0
    if which != SCHULZ_START:  # the start is one scaled copy per block: no conflicts
        assert rep[2] > 0


@pytest.mark.parametrize("which,least", [(FACTOR, 0.5), (SOLVE, 0.2), (SCHULZ_APPLY, 1.0)])
def test_dropped_edges_are_reported(lib, which, least):
    """Sampled single-edge removals: each is reported exactly when it leaves
    its two tasks unordered (no edge orders nothing), and at least `least` of
    them are reported."""
    T = _trees(4, 8)
    st, rep = _check(lib, T, which, tile=16)
    assert st == 0
    E = int(rep[9])
    rng = np.random.default_rng(0)
    sample = rng.choice(E, size=min(E, 60), replace=False)
    reported = 0
    for e in sample:
        s, r = _check(lib, T, which, tile=16, drop=int(e))
        assert s in (0, 9) and r[9] == E - 1
        if s == 9:
            reported += 1
            assert r[10] == 0 and r[3] > 0  # the pair lost its order
            assert 0 <= r[4] < r[5]
        else:
            assert r[10] == 1, e  # unreported only when another path orders the pair
    assert reported >= least * len(sample), (reported, len(sample))


def test_bad_arguments(lib):
    p, C, B = _trees(3, 16)
    rep = np.zeros(11, np.int64)
    assert lib.hlu_debug_check_hazards(len(C), C.ctypes.data, len(B), B.ctypes.data, 32, 0, 16, 5, -1,
                                       rep.ctypes.data) == 1
    assert lib.hlu_debug_check_hazards(len(C), C.ctypes.data, len(B), B.ctypes.data, 32, 0, 17, 0, -1,
                                       rep.ctypes.data) == 1
    assert lib.hlu_debug_check_hazards(len(C), C.ctypes.data, len(B), B.ctypes.data, 32, 0, 16, 0, 1 << 40,
                                       rep.ctypes.data) == 1
    assert lib.hlu_debug_check_hazards(len(C), C.ctypes.data, len(B), B.ctypes.data, 32, 0, 16, 0, -1, None) == 1

"""Brute-force pins of the oracle's cluster and block trees (no GPU)."""
import numpy as np
import pytest

from oracle import mesh as M
from oracle import trees as T


def _setup(n, leaf, eta=2.0):
    m = M.interior_edges(n)
    pts = T.edge_midpoints2(m)
    perm, cl, bl = T.build_trees(m, leaf, eta)
    return m, pts, perm, cl, bl


@pytest.mark.parametrize("n,leaf", [(2, 4), (3, 8), (4, 16), (4, 32), (6, 32)])
def test_cluster_tree_invariants(n, leaf):
    m, pts, perm, cl, bl = _setup(n, leaf)
    N = len(pts)
    assert sorted(perm.tolist()) == list(range(N))
    assert cl[0]["offset"] == 0 and cl[0]["size"] == N
    for cid, c in enumerate(cl):
        idx = perm[c["offset"]:c["offset"] + c["size"]]
        p = pts[idx]
        assert np.array_equal(p.min(0), c["lo"]) and np.array_equal(p.max(0), c["hi"])
        if c["size"] <= leaf:
            assert not c["sons"]
            # stable partitions from the identity order leave every leaf's
            # original DOF indices ascending
            assert np.all(np.diff(idx) > 0)
            continue
        s0, s1 = (cl[s] for s in c["sons"])
        assert s0["offset"] == c["offset"] and s1["offset"] == c["offset"] + s0["size"]
        assert s0["size"] + s1["size"] == c["size"] and s0["size"] > 0 and s1["size"] > 0
        ext = c["hi"] - c["lo"]
        ax = int(np.argmax(ext))
        assert ext[ax] == ext.max() and all(ext[a] < ext[ax] for a in range(ax))
        mid2 = c["lo"][ax] + c["hi"][ax]
        pl = pts[perm[s0["offset"]:s0["offset"] + s0["size"]]]
        pr = pts[perm[s1["offset"]:s1["offset"] + s1["size"]]]
        assert np.all(2 * pl[:, ax] < mid2) and np.all(2 * pr[:, ax] >= mid2)
        # the split sends every point of the cluster to exactly one son
        assert len(pl) + len(pr) == len(idx)
        assert s0["level"] == c["level"] + 1 and s0["parent"] == cid
        # DFS pre-order ids
        assert c["sons"][0] == cid + 1


def test_partition_is_stable():
    m, pts, perm, cl, bl = _setup(4, 16)
    # the permutation inside each son keeps the order the parent had
    def order_in(c):
        return perm[c["offset"]:c["offset"] + c["size"]].tolist()
    for c in cl:
        if not c["sons"]:
            continue
        parent = order_in(c)
        pos = {v: i for i, v in enumerate(parent)}
        for s in c["sons"]:
            child = order_in(cl[s])
            assert all(pos[a] < pos[b] for a, b in zip(child, child[1:]))


@pytest.mark.parametrize("n,leaf,eta", [(2, 4, 2.0), (3, 8, 2.0), (4, 16, 2.0), (4, 8, 1.0), (6, 32, 2.0)])
def test_block_tree_tiles_and_admissibility(n, leaf, eta):
    m, pts, perm, cl, bl = _setup(n, leaf, eta)
    N = len(pts)
    cover = np.zeros((N, N), dtype=np.int32)
    for b in bl:
        r, c = cl[b["row"]], cl[b["col"]]
        if b["kind"] == T.SUB:
            assert len(b["sons"]) == 4 and r["sons"] and c["sons"]
            exp = [(ri, ci) for ri in r["sons"] for ci in c["sons"]]
            got = [(bl[s]["row"], bl[s]["col"]) for s in b["sons"]]
            assert got == exp
            continue
        cover[r["offset"]:r["offset"] + r["size"], c["offset"]:c["offset"] + c["size"]] += 1
        # float geometry (physical units) gives the same decision
        pr = pts[perm[r["offset"]:r["offset"] + r["size"]]] / (2.0 * n)
        pc = pts[perm[c["offset"]:c["offset"] + c["size"]]] / (2.0 * n)
        lo_r, hi_r, lo_c, hi_c = pr.min(0), pr.max(0), pc.min(0), pc.max(0)
        diam = min(np.linalg.norm(hi_r - lo_r), np.linalg.norm(hi_c - lo_c))
        gap = np.maximum(0, np.maximum(lo_c - hi_r, lo_r - hi_c))
        dist = np.linalg.norm(gap)
        if b["kind"] == T.ADM:
            assert dist > 0 and diam <= eta * dist * (1 + 1e-12)
        else:
            assert not r["sons"] or not c["sons"]
            assert dist == 0 or diam > eta * dist * (1 - 1e-12)
    assert cover.min() == 1 and cover.max() == 1


def test_export_layout():
    m, pts, perm, cl, bl = _setup(3, 8)
    p, C, B = T.export_arrays(perm, cl, bl)
    assert C.shape == (len(cl), 12) and B.shape == (len(bl), 8)
    for i, b in enumerate(bl):
        for j, s in enumerate(b["sons"]):
            assert B[i, 3 + j] == s and B[s, 7] == i

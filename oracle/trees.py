"""Geometric cluster tree and eta-admissible block tree (oracle; test
infrastructure only).  Integer-exact: the GPU path must reproduce these arrays
bit for bit.

Paper: H-matrices are defined on a block partition P obtained from a clustering
(Sec. 3); blocks (tau, sigma) that are admissible are stored as X Y^H of rank r
(Definition 1); the cluster tree is geometrically balanced (Sec. 4, after
Grasedyck-Hackbusch 2004) and the admissibility parameter is eta = 2 (Sec. 4).
Sec. 3 announces the eta-admissibility definition but never states it.

Readings:
  * points: doubled-integer edge midpoints p = lattice(lo) + lattice(hi);
  * a cluster holds a contiguous range [offset, offset+size) of the permuted
    DOF order and the tight integer bounding box [lo, hi] of its points;
  * split axis = argmax(hi - lo), ties to the lowest axis; a point goes left iff
    2 p[ax] < lo[ax] + hi[ax]; the partition is stable; a cluster is a leaf iff
    size <= leaf; sons are (left, right); cluster ids are DFS pre-order;
  * admissible iff min(diam^2 tau, diam^2 sigma) <= eta^2 dist^2(tau, sigma) on the
    integer boxes, with eta^2 exact (eta = 2 -> 4); dist = 0 is never admissible;
  * not admissible and (tau or sigma a leaf) -> dense leaf block; otherwise the
    block has the four sons (t0,s0),(t0,s1),(t1,s0),(t1,s1); blocks are listed in
    DFS pre-order.

Pins (tests/test_oracle_trees.py): brute force on small meshes - perm is a
permutation, sons partition parents, boxes are tight, leaf blocks tile N x N
exactly once, every low-rank block passes the test and every dense block has a
leaf cluster.
"""
import numpy as np

ADM, DENSE, SUB = 0, 1, 2


def edge_midpoints2(mesh):
    """Tree points: doubled lattice midpoints on the Kuhn cube, the quantized
    midpoints of a general mesh (mesh.general_mesh)."""
    if "points" in mesh:
        return mesh["points"]
    lat = mesh["lattice"]
    e = mesh["edges"]
    return lat[e[:, 0]] + lat[e[:, 1]]


def cluster_tree(points, leaf):
    """points int64[N, 3].  Returns (perm int64[N], clusters list of dicts with
    keys offset, size, lo, hi, sons, level, parent), ids in DFS pre-order.
    perm[i] = original DOF at permuted position i."""
    N = len(points)
    perm = np.arange(N, dtype=np.int64)
    clusters = []

    def build(offset, size, level, parent):
        cid = len(clusters)
        idx = perm[offset:offset + size]
        pts = points[idx]
        lo = pts.min(axis=0) if size else np.zeros(3, dtype=np.int64)
        hi = pts.max(axis=0) if size else np.zeros(3, dtype=np.int64)
        c = {"offset": offset, "size": size, "lo": lo.copy(), "hi": hi.copy(),
             "sons": [], "level": level, "parent": parent}
        clusters.append(c)
        if size <= leaf:
            return cid
        ext = hi - lo
        ax = int(np.argmax(ext))  # first maximum -> lowest axis on ties
        left = 2 * pts[:, ax] < lo[ax] + hi[ax]
        new = np.concatenate([idx[left], idx[~left]])  # stable partition
        perm[offset:offset + size] = new
        nl = int(left.sum())
        s0 = build(offset, nl, level + 1, cid)
        s1 = build(offset + nl, size - nl, level + 1, cid)
        c["sons"] = [s0, s1]
        return cid

    build(0, N, 0, -1)
    return perm, clusters


def diam2(c):
    d = c["hi"] - c["lo"]
    return int(np.dot(d, d))


def dist2(a, b):
    g = np.maximum(0, np.maximum(b["lo"] - a["hi"], a["lo"] - b["hi"]))
    return int(np.dot(g, g))


def admissible(a, b, eta2):
    d2 = dist2(a, b)
    if d2 == 0:
        return False
    return min(diam2(a), diam2(b)) <= eta2 * d2


def block_tree(clusters, eta2):
    """Returns list of blocks (dicts: row, col, kind, sons), DFS pre-order, with
    kind ADM (low rank leaf), DENSE (dense leaf) or SUB (four sons)."""
    blocks = []

    def build(t, s):
        bid = len(blocks)
        b = {"row": t, "col": s, "kind": None, "sons": []}
        blocks.append(b)
        ct, cs = clusters[t], clusters[s]
        if admissible(ct, cs, eta2):
            b["kind"] = ADM
        elif not ct["sons"] or not cs["sons"]:
            b["kind"] = DENSE
        else:
            b["kind"] = SUB
            for ti in ct["sons"]:
                for si in cs["sons"]:
                    b["sons"].append(build(ti, si))
        return bid

    build(0, 0)
    return blocks


def build_trees(mesh, leaf, eta):
    """Cluster and block trees of the mesh's interior edges.  eta must be such
    that eta^2 is an integer (eta = 2 -> 4)."""
    eta2 = int(round(eta * eta))
    if abs(eta2 - eta * eta) > 1e-12:
        raise ValueError("eta^2 must be an integer")
    perm, clusters = cluster_tree(edge_midpoints2(mesh), leaf)
    blocks = block_tree(clusters, eta2)
    return perm, clusters, blocks


def export_arrays(perm, clusters, blocks):
    """Flat int arrays in the library's export layout.
    clusters: int32[nc, 12] = offset, size, lo[3], hi[3], son0, son1, level, parent
    blocks:   int32[nb, 8]  = row, col, kind, son0..son3, parent
    (son = -1 when absent)."""
    C = np.full((len(clusters), 12), -1, dtype=np.int64)
    for i, c in enumerate(clusters):
        C[i, 0] = c["offset"]
        C[i, 1] = c["size"]
        C[i, 2:5] = c["lo"]
        C[i, 5:8] = c["hi"]
        if c["sons"]:
            C[i, 8], C[i, 9] = c["sons"]
        C[i, 10] = c["level"]
        C[i, 11] = c["parent"]
    B = np.full((len(blocks), 8), -1, dtype=np.int64)
    parent = [-1] * len(blocks)
    for i, b in enumerate(blocks):
        for s in b["sons"]:
            parent[s] = i
    for i, b in enumerate(blocks):
        B[i, 0], B[i, 1], B[i, 2] = b["row"], b["col"], b["kind"]
        for j, s in enumerate(b["sons"]):
            B[i, 3 + j] = s
        B[i, 7] = parent[i]
    return perm.astype(np.int32), C.astype(np.int32), B.astype(np.int32)

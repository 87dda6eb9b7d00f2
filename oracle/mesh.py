"""Kuhn-cube tetrahedral mesh and interior-edge numbering (oracle; test
infrastructure only).

Paper: Sec. 2.1 asks for a conforming, shape-regular, quasi-uniform simplicial
mesh and one degree of freedom per *interior* edge (the basis is fixed by
sigma(Phi_i, e_j) = delta_ij on interior edges; boundary edges carry the PEC
condition E x n = 0 and are eliminated).  Sec. 4 / Example 1 uses the unit cube
cut into 6 tetrahedra and refined.

Readings (the paper leaves these open):
  * mesh: the unit cube split into n^3 sub-cubes, each cut into 6 tetrahedra
    along the 6 permutations of the coordinate axes (Kuhn / Freudenthal split);
  * vertex id v = (i(n+1)+j)(n+1)+k for lattice point (i,j,k), coords (i,j,k)/n;
  * an edge is oriented from its lower to its higher vertex id;
  * an edge is a boundary edge iff both end points lie on one face of the cube;
  * interior edges are numbered in increasing (lo vertex, hi vertex) order.

Pins: the total edge count equals the N_dof column of Table 1 at refinement
levels whose entries are self-consistent; Euler characteristic V - E + F - T = 1;
interior count 7n^3 - 9n^2 + 3n (tests/test_oracle_mesh.py).
"""
import itertools

import numpy as np


def vertex_id(i, j, k, n):
    """Lattice point (i, j, k) of the n-cube -> global vertex id."""
    return (i * (n + 1) + j) * (n + 1) + k


def kuhn_cube(n):
    """Kuhn split of [0,1]^3 into 6 n^3 tetrahedra.

    Returns (lattice, tets): lattice int64[(n+1)^3, 3] integer coordinates
    (the physical coordinates are lattice / n), tets int64[6 n^3, 4] vertex ids.
    Tet of sub-cube c and axis permutation p: c, c+e_p0, c+e_p0+e_p1, c+(1,1,1).
    """
    idx = np.arange(n + 1)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    lattice = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.int64)
    tets = []
    unit = np.eye(3, dtype=np.int64)
    for i in range(n):
        for j in range(n):
            for k in range(n):
                c = np.array([i, j, k], dtype=np.int64)
                for perm in itertools.permutations(range(3)):
                    p0 = c
                    p1 = p0 + unit[perm[0]]
                    p2 = p1 + unit[perm[1]]
                    p3 = p2 + unit[perm[2]]
                    tets.append([vertex_id(*p, n) for p in (p0, p1, p2, p3)])
    return lattice, np.array(tets, dtype=np.int64)


def all_edges(tets):
    """Every distinct tetrahedron edge as a sorted (lo, hi) vertex pair."""
    pairs = set()
    for t in tets:
        for a in range(4):
            for b in range(a + 1, 4):
                u, v = int(t[a]), int(t[b])
                pairs.add((min(u, v), max(u, v)))
    return sorted(pairs)


def all_faces(tets):
    faces = set()
    for t in tets:
        for f in itertools.combinations(sorted(int(x) for x in t), 3):
            faces.add(f)
    return faces


def is_boundary_edge(lattice, n, lo, hi):
    """Both end points on one face x_a = 0 or x_a = n of the cube."""
    a, b = lattice[lo], lattice[hi]
    for ax in range(3):
        for val in (0, n):
            if a[ax] == val and b[ax] == val:
                return True
    return False


def interior_edges(n):
    """Mesh plus its interior edges.

    Returns dict with lattice, coords (lattice / n), tets, edges int64[N, 2]
    (lo, hi) in DOF order, edge_index: {(lo, hi): dof} and boundary_vertex
    (bool per vertex: on a face of the cube).
    """
    lattice, tets = kuhn_cube(n)
    edges = [e for e in all_edges(tets) if not is_boundary_edge(lattice, n, *e)]
    edges = np.array(edges, dtype=np.int64).reshape(-1, 2)
    edge_index = {(int(e[0]), int(e[1])): d for d, e in enumerate(edges)}
    bv = np.any((lattice == 0) | (lattice == n), axis=1)
    return {"n": n, "lattice": lattice, "coords": lattice.astype(np.float64) / n, "tets": tets, "edges": edges,
            "edge_index": edge_index, "boundary_vertex": bv}


def point_scale(extent):
    """Largest power of two s with 2 extent s <= 2^21 (extent > 0)."""
    s = 1.0
    while 2.0 * extent * s * 2.0 <= 2.0 ** 21:
        s *= 2.0
    while 2.0 * extent * s > 2.0 ** 21:
        s *= 0.5
    return s


def general_mesh(coords, tets):
    """A conforming tetrahedral mesh given by vertex coordinates (float64
    [nv, 3]) and tetrahedra (int [nt, 4] vertex ids), with one degree of
    freedom per interior edge (Sec. 2.1; PEC eliminates the boundary edges).

    Readings: a boundary face belongs to exactly one tetrahedron; a boundary
    edge (and vertex) lies on a boundary face; interior edges are oriented
    from the lower to the higher vertex id and numbered in increasing
    (lo, hi) order, as on the Kuhn cube.  The cluster tree's points are the
    edge midpoints on an integer grid: p = rint((x_lo + x_hi - 2 b) s), b the
    lower corner of the vertices' bounding box and s = point_scale(extent), a
    power of two, so every step is an exactly reproducible IEEE operation.

    Returns the dict of interior_edges with n = 0 and no lattice, plus points
    (int64 [N, 3]), the tree points in DOF order.
    """
    coords = np.asarray(coords, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    count = {}
    for t in tets:
        for f in itertools.combinations(sorted(int(x) for x in t), 3):
            count[f] = count.get(f, 0) + 1
    bfaces = [f for f, c in count.items() if c == 1]
    bedges = set()
    bv = np.zeros(len(coords), dtype=bool)
    for f in bfaces:
        for a, b in itertools.combinations(f, 2):
            bedges.add((a, b))
        bv[list(f)] = True
    edges = [e for e in all_edges(tets) if e not in bedges]
    edges = np.array(edges, dtype=np.int64).reshape(-1, 2)
    edge_index = {(int(e[0]), int(e[1])): d for d, e in enumerate(edges)}
    lo = coords.min(axis=0)
    extent = float((coords.max(axis=0) - lo).max())
    s = point_scale(extent)
    mid = ((coords[edges[:, 0]] + coords[edges[:, 1]]) - 2.0 * lo) * s
    points = np.rint(mid).astype(np.int64)
    return {"n": 0, "coords": coords, "tets": tets, "edges": edges, "edge_index": edge_index,
            "boundary_vertex": bv, "points": points}


def n_interior_edges_formula(n):
    return 7 * n ** 3 - 9 * n ** 2 + 3 * n


def n_total_edges_formula(n):
    return 3 * n * (n + 1) ** 2 + 3 * n ** 2 * (n + 1) + n ** 3

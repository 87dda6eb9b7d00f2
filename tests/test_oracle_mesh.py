"""Pins of the oracle's Kuhn mesh and interior-edge numbering (no GPU)."""
import os

import numpy as np
import pytest

from oracle import mesh as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    for line in open(os.path.join(GOLDEN, "table1_ndof.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, ndof, ok = (int(x) for x in line.split())
        rows.append((k, ndof, ok))
    return rows


def test_table1_ndof_is_total_edge_count():
    # Table 1 N_dof at k = 2, 3, 6 equals the total edge count at n = 2^(k-1)
    for k, ndof, ok in _table1():
        n = 2 ** (k - 1)
        if ok:
            assert M.n_total_edges_formula(n) == ndof
        else:
            assert M.n_total_edges_formula(n) != ndof


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_edge_counts_brute_force(n):
    lattice, tets = M.kuhn_cube(n)
    edges = M.all_edges(tets)
    assert len(edges) == M.n_total_edges_formula(n)
    inner = M.interior_edges(n)["edges"]
    assert len(inner) == M.n_interior_edges_formula(n)
    # Table 1: n = 2 (k = 2) has 98 edges, n = 4 (k = 3) has 604
    if n == 2:
        assert len(edges) == 98
    if n == 4:
        assert len(edges) == 604


@pytest.mark.parametrize("n", [1, 2, 3])
def test_euler_characteristic(n):
    lattice, tets = M.kuhn_cube(n)
    V = len(lattice)
    E = len(M.all_edges(tets))
    F = len(M.all_faces(tets))
    T = len(tets)
    assert V - E + F - T == 1


@pytest.mark.parametrize("n", [2, 3])
def test_kuhn_conforming_and_volume(n):
    lattice, tets = M.kuhn_cube(n)
    P = lattice[tets].astype(float) / n
    vols = np.abs(np.linalg.det(np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0],
                                          P[:, 3] - P[:, 0]], axis=2))) / 6.0
    assert np.allclose(vols, 1.0 / (6 * n ** 3))
    assert abs(vols.sum() - 1.0) < 1e-12
    # every face is shared by 1 (boundary) or 2 (interior) tetrahedra
    count = {}
    for t in tets:
        s = sorted(int(x) for x in t)
        for f in ((s[0], s[1], s[2]), (s[0], s[1], s[3]), (s[0], s[2], s[3]), (s[1], s[2], s[3])):
            count[f] = count.get(f, 0) + 1
    assert set(count.values()) <= {1, 2}
    nb = sum(1 for v in count.values() if v == 1)
    assert nb == 12 * n * n  # 6 faces x n^2 squares x 2 triangles


def test_interior_edges_sorted_and_oriented():
    m = M.interior_edges(3)
    e = m["edges"]
    assert np.all(e[:, 0] < e[:, 1])
    keys = e[:, 0] * 10 ** 6 + e[:, 1]
    assert np.all(np.diff(keys) > 0)
    lat = m["lattice"]
    for lo, hi in e:
        for ax in range(3):
            for val in (0, 3):
                assert not (lat[lo, ax] == val and lat[hi, ax] == val)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_general_mesh_reproduces_the_kuhn_lattice_rules(n):
    """Given the Kuhn cube as plain coordinates and tetrahedra, the general
    rule (a boundary face belongs to one tetrahedron, boundary edges and
    vertices lie on boundary faces) selects exactly the edges and vertices the
    lattice rule (both end points on one face of the cube) selects."""
    import synth
    coords, tets = synth.perturbed_kuhn_mesh(n, 0.0, 1)
    g = M.general_mesh(coords, tets)
    m = M.interior_edges(n)
    assert np.array_equal(g["edges"], m["edges"])
    assert np.array_equal(g["boundary_vertex"], m["boundary_vertex"])
    assert len(g["edges"]) == M.n_interior_edges_formula(n)


def test_general_mesh_points_are_exact_quantised_midpoints():
    import synth
    coords, tets = synth.perturbed_kuhn_mesh(3, 0.2, 7)
    g = M.general_mesh(coords, tets)
    lo = coords.min(axis=0)
    extent = (coords.max(axis=0) - lo).max()
    s = M.point_scale(extent)
    assert s == 2.0 ** 20 and 2 * extent * s <= 2 ** 21  # unit cube
    mid = coords[g["edges"][:, 0]] + coords[g["edges"][:, 1]] - 2 * lo
    assert np.abs(g["points"] - mid * s).max() <= 0.5
    assert g["points"].min() >= 0 and g["points"].max() <= 2 ** 21


def test_perturbed_mesh_is_valid():
    """No tetrahedron of the perturbed cube inverts (each keeps the
    orientation it has on the lattice, which alternates with the parity of
    its axis permutation), the tetrahedra still tile the unit cube (volumes
    sum to 1) and the Euler characteristic is 1."""
    import synth

    def signed(coords, tets):
        P = coords[tets]
        return np.einsum("ti,ti->t", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0])) / 6.0

    c0, t0 = synth.perturbed_kuhn_mesh(4, 0.0, 3)
    coords, tets = synth.perturbed_kuhn_mesh(4, 0.2, 3)
    v0, v = signed(c0, t0), signed(coords, tets)
    assert np.all(np.sign(v) == np.sign(v0)) and np.abs(v).min() > 0
    assert abs(np.abs(v).sum() - 1.0) < 1e-12
    V, E, F, T = len(coords), len(M.all_edges(tets)), len(M.all_faces(tets)), len(tets)
    assert V - E + F - T == 1

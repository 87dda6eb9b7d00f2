"""Pins of the oracle's Nedelec assembly and load vector (no GPU)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import fem as F
from oracle import mesh as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_reference_tet_by_hand():
    P = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], dtype=float)
    g = np.array([[0, 1, 2, 3]])
    Ke, Me = F.element_matrices(P, g)
    for line in open(os.path.join(GOLDEN, "reference_tet.txt")):
        if line.startswith("#") or not line.strip():
            continue
        which, r, c, v = line.split()
        mat = Ke[0] if which == "K" else Me[0]
        assert abs(mat[int(r), int(c)] - float(v)) < 1e-15
        assert abs(mat[int(c), int(r)] - float(v)) < 1e-15


def test_tangential_moment_is_one():
    # sigma(Phi_i, e_j) = delta_ij: the tangential integral of w_ab along edge a->b is 1,
    # and 0 along the other edges (checked with a 5-point Gauss rule on each edge)
    P = np.array([[0.1, 0.2, 0.0], [1.0, 0.3, 0.2], [0.2, 1.1, 0.1], [0.3, 0.1, 0.9]])
    G, vol = F.barycentric_gradients(P[None])
    G = G[0]
    xg, wg = np.polynomial.legendre.leggauss(5)
    s = 0.5 * (xg + 1.0)
    w = 0.5 * wg
    for (a, b) in F.LOCAL_EDGES:
        for (c, d) in F.LOCAL_EDGES:
            tang = P[d] - P[c]
            tot = 0.0
            for si, wi in zip(s, w):
                lam = np.zeros(4)
                lam[c], lam[d] = 1.0 - si, si
                phi = lam[a] * G[b] - lam[b] * G[a]
                tot += wi * phi.dot(tang)
            assert abs(tot - (1.0 if (a, b) == (c, d) else 0.0)) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 4])
def test_de_rham_gradients_in_kernel(n):
    m = M.interior_edges(n)
    K, Mm = F.assemble(m, 1.0, parts=True)
    G = F.gradient_matrix(m)
    assert G.shape[1] == (n - 1) ** 3
    KG = K @ G
    assert abs(KG).max() < 1e-12 * abs(K).max()
    assert abs(Mm @ G).max() > 1e-3 * abs(Mm).max()


def test_symmetry_spd_and_nullspace():
    n = 3
    m = M.interior_edges(n)
    K, Mm = F.assemble(m, 1.0, parts=True)
    assert abs(K - K.T).max() < 1e-14
    assert abs(Mm - Mm.T).max() < 1e-15
    np.linalg.cholesky(Mm.toarray())  # M is SPD
    ev = np.linalg.eigvalsh(K.toarray())
    nz = np.sum(ev < 1e-10 * ev.max())
    assert nz == (n - 1) ** 3
    assert ev.min() > -1e-10 * ev.max()


def test_cavity_eigenvalues():
    # Maxwell eigenvalues of the unit cube: pi^2 (l^2+m^2+n^2), at least two indices
    # nonzero: 2 pi^2 (x3), 3 pi^2 (x2).  Discrete values converge as n grows.
    errs = []
    for n in (3, 5):
        m = M.interior_edges(n)
        K, Mm = F.assemble(m, 1.0, parts=True)
        ev = sla.eigh(K.toarray(), Mm.toarray(), eigvals_only=True)
        ev = ev[ev > 1e-8 * ev.max()]
        ev = np.sort(ev)[:5]
        exact = np.pi ** 2 * np.array([2, 2, 2, 3, 3])
        errs.append(np.abs(ev - exact) / exact)
    assert np.all(errs[1] < 0.08)
    assert errs[1].max() < errs[0].max()


def test_manufactured_boundary_and_field():
    x = np.random.default_rng(1).random((50, 3))
    E = F.manufactured_E(x)
    # E x n = 0 on x = 0 (n = -e_x): tangential components E_y, E_z vanish
    x0 = x.copy(); x0[:, 0] = 0.0
    E0 = F.manufactured_E(x0)
    assert np.abs(E0[:, 1:]).max() < 1e-15
    # curl curl E = 2 pi^2 E via finite differences of curl
    h = 1e-4

    def curl(f, p):
        J = np.zeros((3, 3))
        for j in range(3):
            e = np.zeros(3); e[j] = h
            J[:, j] = (f(p + e) - f(p - e)) / (2 * h)
        return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])

    p = np.array([0.3, 0.6, 0.2])
    cc = curl(lambda q: curl(lambda r: F.manufactured_E(r[None])[0], q), p)
    assert np.allclose(cc, 2 * np.pi ** 2 * F.manufactured_E(p[None])[0], rtol=1e-4)


def test_manufactured_convergence_rate():
    kappa = 1.0
    errs = []
    for n in (4, 8, 16):
        m = M.interior_edges(n)
        A = F.assemble(m, kappa)
        b = F.manufactured_rhs(m, kappa)
        x = spla.spsolve(A.tocsc(), b)
        errs.append(F.l2_error(m, x, F.manufactured_E))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert 0.85 < rates[0] < 1.3 and 0.9 < rates[1] < 1.2, (errs, rates)


@pytest.mark.parametrize("n", [2, 3, 4])
@pytest.mark.parametrize("J", [(0.0, 0.0, 1.0), (1.0, -2.0, 0.5)])
def test_constant_current_rhs_is_discretely_divergence_free(n, J):
    """For a constant J, <J, grad phi_v> = -<div J, phi_v> = 0 for every
    interior vertex hat function phi_v (zero on the boundary), and grad phi_v
    is the combination G[:, v] of interior edge basis functions, so
    G^T b = 0 up to rounding."""
    m = M.interior_edges(n)
    b = F.constant_current_rhs(m, J)
    G = F.gradient_matrix(m)
    assert np.abs(G.T @ b).max() <= 1e-14 * max(1.0, np.abs(b).max())
    assert np.abs(b).max() > 0.01 / n ** 3


def test_constant_current_rhs_equals_exact_element_integrals():
    """The integral of a barycentric coordinate over a tetrahedron is |T|/4,
    so b_e = sum over the tets of e of |T|/4 J . (grad l_hi - grad l_lo); the
    gradients here come from inverting [1 x y z] at the four vertices."""
    n, J = 2, np.array([0.0, 0.0, 1.0])
    m = M.interior_edges(n)
    b = F.constant_current_rhs(m, J)
    lat = m["lattice"] / float(n)
    index = {(int(a), int(c)): e for e, (a, c) in enumerate(m["edges"])}
    ref = np.zeros(len(m["edges"]))
    for tet in m["tets"]:
        V = np.hstack([np.ones((4, 1)), lat[tet]])
        vol = abs(np.linalg.det(V)) / 6.0
        grads = np.linalg.inv(V)[1:, :].T  # row i: grad of the barycentric coordinate of vertex i
        for i in range(4):
            for j in range(i + 1, 4):
                a, c = (i, j) if tet[i] < tet[j] else (j, i)
                e = index.get((int(tet[a]), int(tet[c])))
                if e is not None:
                    ref[e] += vol / 4.0 * J @ (grads[c] - grads[a])
    assert np.abs(b - ref).max() <= 1e-15 * 10 + 1e-14 * np.abs(ref).max()


def test_general_mesh_de_rham_symmetry_and_nullspace():
    """On a perturbed (non-lattice) mesh the assembled K annihilates the
    gradients of the interior vertex functions (the discrete de Rham
    property holds on any mesh), K and M are symmetric, M is SPD and the null
    space of K has the dimension of the interior vertices."""
    import synth
    coords, tets = synth.perturbed_kuhn_mesh(3, 0.2, 11)
    m = M.general_mesh(coords, tets)
    K, Mm = F.assemble(m, 1.0, parts=True)
    G = F.gradient_matrix(m)
    assert G.shape[1] == 8  # (n - 1)^3 interior vertices
    assert abs(K @ G).max() < 1e-12 * abs(K).max()
    assert abs(K - K.T).max() < 1e-13 * abs(K).max() and abs(Mm - Mm.T).max() < 1e-15
    ev_m = sla.eigvalsh(Mm.toarray())
    assert ev_m.min() > 0
    ev_k = sla.eigvalsh(K.toarray(), Mm.toarray())
    assert int(np.sum(np.abs(ev_k) < 1e-8)) == G.shape[1]


def test_material_coefficient_keeps_gradients_in_kernel():
    """curl(beta^-1 curl): a per-element beta scales only the curl-curl part,
    so discrete gradients stay in its kernel and the mass matrix is unchanged
    (Sec. 2, the operator with the material coefficient)."""
    n = 4
    m = M.interior_edges(n)
    rng = np.random.default_rng(5)
    beta = rng.uniform(1.0, 10.0, size=6 * n ** 3)
    K1, M1 = F.assemble(m, 1.0, parts=True)
    Kb, Mb = F.assemble(m, 1.0, parts=True, beta=beta)
    G = F.gradient_matrix(m)
    assert abs(Kb @ G).max() < 1e-12 * abs(Kb).max()
    assert abs(Mb - M1).max() == 0.0
    assert abs(Kb - K1).max() > 1e-3 * abs(K1).max()
    A = F.assemble(m, 2.0, beta=beta)
    assert abs(A - (Kb - 4.0 * Mb)).max() < 1e-14 * abs(A).max()
    with pytest.raises(ValueError):
        F.assemble(m, 1.0, beta=np.zeros(6 * n ** 3))


def test_constant_beta_divides_the_cavity_eigenvalues():
    """beta = c everywhere: the cavity eigenvalues pi^2 (l^2 + m^2 + n^2) / c
    (at least two indices nonzero) - the first, 2 pi^2 / c, three times."""
    c = 4.0
    for n in (3, 5):
        m = M.interior_edges(n)
        Kb, Mm = F.assemble(m, 1.0, parts=True, beta=np.full(6 * n ** 3, c))
        ev = sla.eigh(Kb.toarray(), Mm.toarray(), eigvals_only=True)
        ev = np.sort(ev[ev > 1e-8 * ev.max()])[:5]
        exact = np.pi ** 2 * np.array([2, 2, 2, 3, 3]) / c
        err = np.abs(ev - exact) / exact
    assert np.all(err < 0.08)


def test_magnet_occupies_its_volume():
    """Example 3's magnet (0.5 x 0.5 x 0.75, centred): at n = 8 the lattice
    fits its faces, so exactly 0.1875 of the 3,072 tetrahedra (576) lie in it,
    each with all four vertices in the closed box."""
    n = 8
    m = M.interior_edges(n)
    beta = F.magnet_beta(m, 10.0)
    inside = beta == 10.0
    assert inside.sum() == 576 and np.all((beta == 1.0) | inside)
    P = m["coords"][m["tets"][inside]]
    for a, (lo, hi) in enumerate(F.MAGNET_BOX):
        assert np.all(P[:, :, a] >= lo - 1e-15) and np.all(P[:, :, a] <= hi + 1e-15)

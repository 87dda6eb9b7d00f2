"""Lowest-order Nedelec (first kind) edge elements: element matrices, CSR
assembly of A = K - kappa^2 M, and the load vector (oracle; test infrastructure
only).

Paper: the operator curl(beta^-1 curl E) - kappa E = J_S with PEC (Sec. 2,
second-order form), the bilinear form a(E,Phi) = <curl E, curl Phi> - kappa <E,Phi>
(Sec. 2.1, weak form, beta = 1), the local space N_0(T) = {a + b x x}, the edge
basis sigma(Phi_i, e_j) = delta_ij, A_ij = a(Phi_i, Phi_j) and b_j = <J_S, Phi_j>
(Sec. 2.1, stiffness-matrix equation).

Readings:
  * the paper's kappa (= omega^2 zeta) is written here as kappa^2 with kappa a
    wave number, so A = K - kappa^2 M (paper-kappa = kappa^2);
  * basis on edge (a, b), a the lower global vertex id: w = l_a grad l_b - l_b grad l_a
    (Whitney form; its tangential integral from a to b is exactly 1), so
    curl w = 2 grad l_a x grad l_b;
  * int_T l_i l_j = |T| (1 + delta_ij) / 20 (exact for linear barycentrics);
  * load vector: 4-point degree-2 tetrahedron rule, barycentric points
    (alpha, alpha, alpha, beta) and permutations, alpha = (5 - sqrt 5)/20,
    beta = (5 + 3 sqrt 5)/20, weights |T|/4;
  * manufactured field E = (sin pi y sin pi z, sin pi z sin pi x, sin pi x sin pi y):
    div E = 0 and curl curl E = 2 pi^2 E, so J = (2 pi^2 - kappa^2) E, and
    E x n = 0 on the cube's boundary;
  * Example 1's source J_S = [0, 0, 1]^T is a constant current density
    (constant_current_rhs);
  * the material coefficient beta is constant on each tetrahedron and scales
    that element's curl-curl matrix by 1/beta; Example 3's magnet
    (0.5 x 0.5 x 0.75 in the unit box, beta = 10, air beta = 1) is read as
    centred in the box (magnet_beta);
  * with conductivity chi > 0 the paper's kappa = omega^2 (alpha + i chi/omega)
    is complex and enters as given, A = K_beta - kappa M
    (assemble_time_harmonic): the test functions are not conjugated, so A is
    complex symmetric, A^T = A.

Pins (tests/test_oracle_fem.py): discrete de Rham property C G = 0 and K G = 0;
null space of K of dimension (n-1)^3; cavity eigenvalues 2pi^2 (x3), 3pi^2 (x2);
symmetry; M SPD; reference-tetrahedron element matrices worked by hand; L2
convergence of the manufactured solution at rate ~1; the constant-current load
vector is discretely divergence-free (G^T b = 0) and equals the exact integral
|T|/4 J . (grad l_b - grad l_a) computed element by element; with a material
coefficient, K_beta G = 0 still holds (only the curl-curl part carries beta),
a constant beta = c gives K / c (cavity eigenvalues divided by c), and the
magnet holds 0.1875 of the cube's volume (576 of the 3,072 tetrahedra at n = 8).
The complex assembly reduces to the real one at chi = 0, is symmetric and not
Hermitian, and its solutions obey the energy identities
x^H b = x^H K x - omega^2 alpha x^H M x - i omega chi x^H M x (both forms
real); at a discrete cavity resonance (K v = lambda M v, omega^2 alpha =
lambda) A v = -i omega chi M v exactly, so the conductivity alone keeps A
nonsingular there.
"""
import math

import numpy as np
import scipy.sparse as sp

LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]

QUAD_ALPHA = (5.0 - math.sqrt(5.0)) / 20.0
QUAD_BETA = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0


def quad_points_bary():
    """Barycentric coordinates of the 4-point rule, shape (4, 4)."""
    q = np.full((4, 4), QUAD_ALPHA)
    for i in range(4):
        q[i, i] = QUAD_BETA
    return q


def barycentric_gradients(P):
    """P: (T, 4, 3) vertex coordinates -> (grad lambda (T, 4, 3), |T| (T,))."""
    P = np.asarray(P, dtype=np.float64)
    Jm = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    Jinv = np.linalg.inv(Jm)  # rows are grad lambda_1..3
    G = np.zeros(P.shape)
    G[:, 1:] = Jinv
    G[:, 0] = -Jinv.sum(axis=1)
    vol = np.abs(np.linalg.det(Jm)) / 6.0
    return G, vol


def local_orientation(g):
    """Oriented local edges of each tet: int array (T, 6, 2) of local vertex
    indices (a, b) with global id g[a] < g[b], in LOCAL_EDGES order."""
    g = np.asarray(g)
    out = np.zeros((g.shape[0], 6, 2), dtype=np.int64)
    for r, (p, q) in enumerate(LOCAL_EDGES):
        swap = g[:, p] > g[:, q]
        out[:, r, 0] = np.where(swap, q, p)
        out[:, r, 1] = np.where(swap, p, q)
    return out


def _take(G, idx):
    """G (T, 4, 3), idx (T,) local vertex -> (T, 3)."""
    return G[np.arange(G.shape[0]), idx]


def element_matrices(P, g):
    """Element curl-curl K_e and mass M_e, each (T, 6, 6), of tetrahedra with
    vertex coordinates P (T, 4, 3) and global vertex ids g (T, 4); edges in
    LOCAL_EDGES order with the global lo->hi orientation."""
    G, vol = barycentric_gradients(P)
    E = local_orientation(g)
    T = G.shape[0]
    Ke = np.zeros((T, 6, 6))
    Me = np.zeros((T, 6, 6))

    def mom(i, j):  # int_T lambda_i lambda_j, elementwise over tets
        return vol * (1.0 + (i == j)) / 20.0

    def dot(u, v):
        return np.einsum("ti,ti->t", u, v)

    for r in range(6):
        a, b = E[:, r, 0], E[:, r, 1]
        Ga, Gb = _take(G, a), _take(G, b)
        ca = np.cross(Ga, Gb)
        for s in range(6):
            c, d = E[:, s, 0], E[:, s, 1]
            Gc, Gd = _take(G, c), _take(G, d)
            cc = np.cross(Gc, Gd)
            Ke[:, r, s] = 4.0 * vol * dot(ca, cc)
            Me[:, r, s] = (mom(a, c) * dot(Gb, Gd) - mom(a, d) * dot(Gb, Gc)
                           - mom(b, c) * dot(Ga, Gd) + mom(b, d) * dot(Ga, Gc))
    return Ke, Me


def _tet_data(mesh):
    tets = mesh["tets"]
    return tets, mesh["coords"][tets]


def _tet_dofs(mesh, tets):
    """(T, 6) interior-edge DOF of each local edge, -1 for boundary edges."""
    eidx = mesh["edge_index"]
    dofs = np.full((tets.shape[0], 6), -1, dtype=np.int64)
    for t in range(tets.shape[0]):
        for r, (p, q) in enumerate(LOCAL_EDGES):
            u, v = int(tets[t, p]), int(tets[t, q])
            dofs[t, r] = eidx.get((min(u, v), max(u, v)), -1)
    return dofs


def assemble(mesh, kappa, parts=False, beta=None):
    """CSR matrix A = K - kappa^2 M over interior edges (rows/cols in DOF order,
    columns ascending within a row; the pattern holds every pair of interior
    edges that share a tetrahedron, explicit zeros kept).

    beta (optional, one value per tetrahedron): the material coefficient of
    the curl-curl term, K = sum_T beta_T^-1 K_T (the operator
    curl(beta^-1 curl E) - kappa E of Sec. 2, beta constant on each element);
    None is beta = 1.  parts=True returns (K, M) instead.
    """
    N = len(mesh["edges"])
    tets, P = _tet_data(mesh)
    Ke, Me = element_matrices(P, tets)
    if beta is not None:
        beta = np.asarray(beta, dtype=np.float64).reshape(-1)
        if beta.shape[0] != tets.shape[0] or not np.all(beta > 0):
            raise ValueError("beta: one positive value per tetrahedron")
        Ke = Ke / beta[:, None, None]
    dofs = _tet_dofs(mesh, tets)
    R = np.repeat(dofs[:, :, None], 6, axis=2)
    C = np.repeat(dofs[:, None, :], 6, axis=1)
    keep = (R >= 0) & (C >= 0)
    rows, cols = R[keep], C[keep]
    K = _coo_to_csr(rows, cols, Ke[keep], N)
    M = _coo_to_csr(rows, cols, Me[keep], N)
    if parts:
        return K, M
    A = K.copy()
    A.data = K.data - kappa * kappa * M.data
    return A


def time_harmonic_kappa(omega, alpha, chi):
    """The paper's mass coefficient kappa = omega^2 zeta with
    zeta = alpha + i chi / omega (Sec. 2): alpha the dielectric permeability,
    chi the conductivity, omega the angular frequency."""
    return omega * omega * (alpha + 1j * chi / omega)


def assemble_time_harmonic(mesh, omega, alpha, chi, beta=None):
    """CSR matrix A = K_beta - kappa M with the complex kappa of
    time_harmonic_kappa (the operator curl(beta^-1 curl E) - kappa E of Sec. 2
    with conductivity): complex symmetric, not Hermitian, on the pattern of
    assemble.  chi = 0, alpha = 1 is assemble(mesh, omega)."""
    K, M = assemble(mesh, 0.0, parts=True, beta=beta)
    kap = time_harmonic_kappa(omega, alpha, chi)
    A = K.astype(np.complex128)
    A.data = K.data - kap * M.data
    return A


MAGNET_BOX = ((0.25, 0.75), (0.25, 0.75), (0.125, 0.875))


def magnet_beta(mesh, beta_in=10.0, box=MAGNET_BOX):
    """Per-tetrahedron material coefficient of Example 3 (Sec. 4): a magnet of
    0.5 x 0.5 x 0.75 inside the unit box, read as centred, with beta = beta_in
    there and beta = 1 in the surrounding air; a tetrahedron belongs to the
    magnet when its centroid does."""
    tets, P = _tet_data(mesh)
    c = P.mean(axis=1)
    inside = np.ones(c.shape[0], dtype=bool)
    for a, (lo, hi) in enumerate(box):
        inside &= (c[:, a] > lo) & (c[:, a] < hi)
    return np.where(inside, float(beta_in), 1.0)


def _coo_to_csr(rows, cols, vals, N):
    """Sum duplicates, keep explicit zeros, sort columns in each row."""
    key = rows * N + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uniq, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(vals, start) if len(vals) else vals
    r = uniq // N
    c = uniq % N
    indptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(indptr, r + 1, 1)
    indptr = np.cumsum(indptr)
    return sp.csr_matrix((sums, c, indptr), shape=(N, N))


def _basis_at_quad(G, E, Q):
    """Whitney basis of the 6 oriented edges at the 4 quadrature points:
    (T, 6, 4, 3)."""
    T = G.shape[0]
    out = np.zeros((T, 6, 4, 3))
    for r in range(6):
        a, b = E[:, r, 0], E[:, r, 1]
        la = Q[:, a].T  # (T, 4) lambda_a at the points
        lb = Q[:, b].T
        Ga, Gb = _take(G, a), _take(G, b)
        out[:, r] = la[:, :, None] * Gb[:, None, :] - lb[:, :, None] * Ga[:, None, :]
    return out


def manufactured_E(x):
    """E = (sin pi y sin pi z, sin pi z sin pi x, sin pi x sin pi y); x (..., 3)."""
    s = np.sin(np.pi * x)
    return np.stack([s[..., 1] * s[..., 2], s[..., 2] * s[..., 0], s[..., 0] * s[..., 1]], axis=-1)


def manufactured_J(x, kappa):
    return (2.0 * np.pi ** 2 - kappa * kappa) * manufactured_E(x)


def load_vector(mesh, Jfun):
    """b_j = <J, Phi_j> with the 4-point rule; Jfun maps points (..., 3) -> (..., 3)."""
    N = len(mesh["edges"])
    tets, P = _tet_data(mesh)
    G, vol = barycentric_gradients(P)
    E = local_orientation(tets)
    Q = quad_points_bary()
    X = np.einsum("qv,tvi->tqi", Q, P)  # (T, 4, 3) quadrature points
    Jq = Jfun(X)
    phi = _basis_at_quad(G, E, Q)
    contrib = (vol / 4.0)[:, None] * np.einsum("trqi,tqi->tr", phi, Jq)
    dofs = _tet_dofs(mesh, tets)
    b = np.zeros(N)
    keep = dofs >= 0
    np.add.at(b, dofs[keep], contrib[keep])
    return b


def manufactured_rhs(mesh, kappa):
    return load_vector(mesh, lambda X: manufactured_J(X, kappa))


def constant_current_rhs(mesh, J):
    """b_j = <J_S, Phi_j> for a constant current density J_S (Sec. 4, Example 1
    takes J_S = [0, 0, 1]^T), by the same 4-point rule, which is exact here:
    J_S . Phi_j is linear on every tetrahedron."""
    Jv = np.asarray(J, dtype=float).reshape(3)
    return load_vector(mesh, lambda X: np.broadcast_to(Jv, X.shape))


def l2_error(mesh, x, Efun):
    """sqrt(sum_T int_T |E - E_h|^2) with the 4-point rule, E_h = sum x_j Phi_j."""
    tets, P = _tet_data(mesh)
    G, vol = barycentric_gradients(P)
    E = local_orientation(tets)
    Q = quad_points_bary()
    X = np.einsum("qv,tvi->tqi", Q, P)
    phi = _basis_at_quad(G, E, Q)
    dofs = _tet_dofs(mesh, tets)
    coef = np.where(dofs >= 0, x[np.maximum(dofs, 0)], 0.0)  # (T, 6)
    Eh = np.einsum("tr,trqi->tqi", coef, phi)
    err2 = np.sum((vol / 4.0)[:, None] * np.sum((Efun(X) - Eh) ** 2, axis=2))
    return math.sqrt(err2)


def gradient_matrix(mesh):
    """Discrete gradient G: interior vertices -> interior edges, G[e, v] = +1 if v
    is the head (hi) of e, -1 if the tail (lo).  Interior vertices are those
    on no boundary face, numbered by id."""
    edges, bv = mesh["edges"], mesh["boundary_vertex"]
    inner = [v for v in range(len(bv)) if not bv[v]]
    vpos = {v: i for i, v in enumerate(inner)}
    rows, cols, vals = [], [], []
    for e, (lo, hi) in enumerate(edges):
        if int(hi) in vpos:
            rows.append(e); cols.append(vpos[int(hi)]); vals.append(1.0)
        if int(lo) in vpos:
            rows.append(e); cols.append(vpos[int(lo)]); vals.append(-1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(edges), len(inner)))

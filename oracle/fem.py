"""Lowest-order Nedelec (Whitney) element matrices and global assembly.

Oracle (test infrastructure only).

Paper: Eq. 2.2 (sesquilinear form a_xi(E, v) = int curl E . conj(curl v)
- (k^2 + i xi) int E . conj(v), load F(v) = int F . conj(v)) and Sec. 2.2
(Galerkin matrix (A_xi)_ij = a_xi(w_j, w_i), f_i = F(w_i)).

Readings:
  * basis of the oriented edge (p -> q): w_pq = lam_p grad lam_q - lam_q grad lam_p
    (Whitney form), so the DOF functional int_e w . tau ds equals 1 on its own edge.
  * the basis is real, so A_xi = K - (k^2 + i xi) M with K, M real symmetric
    (K_ij = int curl w_j . curl w_i, M_ij = int w_j . w_i).
  * load-vector quadrature: the conical-product (Duffy) Gauss-Legendre rule with
    q points per direction on the reference tetrahedron (xi_1, xi_2, xi_3 >= 0,
    sum <= 1), xi_1 = u, xi_2 = (1-u) v, xi_3 = (1-u)(1-v) w,
    weight = W_u W_v W_w (1-u)^2 (1-v); reference vertex m <-> path vertex P_m.
    q = 3 is the default (exact for total degree 3).

  * impedance boundary condition (Eq. imp): curl E x n - i sign(xi) k (n x E) x n = 0 on
    the boundary. Integrating curl curl E . v by parts leaves the boundary integral
    int (n x curl E) . v = -i sign(xi) k int E_T . v_T, so
    A_xi = K - (k^2 + i xi) M - i sign(xi) k B, B_ij = int_{boundary} (w_j)_T . (w_i)_T.
    sign(0) is read as +1 (the paper runs the impedance problem with xi = 0; +1 is the
    outgoing condition for the time dependence exp(-i omega t) of Sec. 1.1). On a boundary
    triangle the tangential trace of w_pq is the triangle's own Whitney form
    lam_p grad_F lam_q - lam_q grad_F lam_p (grad_F the surface gradient, the tangential
    part of the tetrahedron's gradient), with int_F lam_i lam_j = |F| (1 + delta_ij) / 12.

Element matrices are computed per tetrahedron from its vertex coordinates
(barycentric gradients by inverting the 4x4 affine system), not from a closed form.
"""
import numpy as np
import scipy.sparse as sp

from .mesh import LOCAL_EDGES


def bary_gradients(P):
    """Gradients of barycentric coordinates and volumes.

    P: [T, 4, 3] vertex coordinates. Returns (G [T, 4, 3], vol [T])."""
    T = P.shape[0]
    Mx = np.ones((T, 4, 4))
    Mx[:, :, 1:] = P
    inv = np.linalg.inv(Mx)  # lam_i(x) = inv[i0] + inv[i,1:] . x  (rows of inv^T)
    # lam = Mx^{-T} [1, x]: lam_i = sum_j inv[j, i] * [1, x]_j
    G = np.transpose(inv[:, 1:, :], (0, 2, 1))  # [T, 4, 3]
    vol = np.abs(np.linalg.det(Mx)) / 6.0
    return G, vol


def element_matrices(P):
    """Whitney curl-curl and mass matrices K_e, M_e [T, 6, 6] for tetrahedra P.

    K_e[a, b] = |T| * 4 (g_p x g_q) . (g_r x g_s) for a = (p, q), b = (r, s);
    M_e[a, b] = int (lam_p g_q - lam_q g_p) . (lam_r g_s - lam_s g_r)
    with int lam_i lam_j = |T| (1 + delta_ij) / 20."""
    G, vol = bary_gradients(P)
    T = P.shape[0]
    K = np.empty((T, 6, 6))
    Mm = np.empty((T, 6, 6))
    mass = lambda i, j: vol * (1.0 + (i == j)) / 20.0
    dot = lambda i, j: np.einsum("ti,ti->t", G[:, i], G[:, j])
    curls = [np.cross(G[:, p], G[:, q]) for p, q in LOCAL_EDGES]
    for a, (p, q) in enumerate(LOCAL_EDGES):
        for b, (r, s) in enumerate(LOCAL_EDGES):
            K[:, a, b] = 4.0 * vol * np.einsum("ti,ti->t", curls[a], curls[b])
            Mm[:, a, b] = (dot(q, s) * mass(p, r) - dot(q, r) * mass(p, s)
                           - dot(p, s) * mass(q, r) + dot(p, r) * mass(q, s))
    return K, Mm


def tet_coords(mesh):
    return mesh.coords(mesh.tets)  # [T, 4, 3]


def assemble_KM(mesh):
    """Global real CSR K, M over the PEC-interior DOFs (Sec. 2.2)."""
    Ke, Me = element_matrices(tet_coords(mesh))
    d = mesh.tet2dof
    rows = np.repeat(d[:, :, None], 6, axis=2)
    cols = np.repeat(d[:, None, :], 6, axis=1)
    keep = (rows >= 0) & (cols >= 0)
    shape = (mesh.n_dof, mesh.n_dof)
    K = sp.coo_matrix((Ke[keep], (rows[keep], cols[keep])), shape=shape).tocsr()
    M = sp.coo_matrix((Me[keep], (rows[keep], cols[keep])), shape=shape).tocsr()
    K.sum_duplicates()
    M.sum_duplicates()
    K.sort_indices()
    M.sort_indices()
    return K, M


def assemble_full_KM(mesh):
    """K, M over all edges (PEC edges kept), indexed like mesh.edges. For tests."""
    Ke, Me = element_matrices(tet_coords(mesh))
    E = mesh.edges.shape[0]
    lut = {(int(a), int(b)): i for i, (a, b) in enumerate(mesh.edges)}
    d = np.empty((mesh.tets.shape[0], 6), dtype=np.int64)
    for k, (a, b) in enumerate(LOCAL_EDGES):
        d[:, k] = [lut[(int(x), int(y))] for x, y in zip(mesh.tets[:, a], mesh.tets[:, b])]
    rows = np.repeat(d[:, :, None], 6, axis=2).ravel()
    cols = np.repeat(d[:, None, :], 6, axis=1).ravel()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(E, E)).tocsr()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(E, E)).tocsr()
    return K, M


FACE_EDGES = [(0, 1), (0, 2), (1, 2)]


def face_matrices(P):
    """Tangential Whitney mass B_F [F, 3, 3] of triangles P [F, 3, 3] (vertex coordinates,
    vertices in increasing id order, edges (0,1), (0,2), (1,2) oriented low -> high).
    Surface gradients from the 2x2 metric of the edge vectors."""
    E = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]], axis=2)  # [F, 3, 2]
    Gm = np.einsum("fia,fib->fab", E, E)
    W = E @ np.linalg.inv(Gm)  # columns: grad lam_1, grad lam_2 (in the plane)
    g1, g2 = W[:, :, 0], W[:, :, 1]
    G = [-(g1 + g2), g1, g2]
    area = 0.5 * np.linalg.norm(np.cross(E[:, :, 0], E[:, :, 1]), axis=1)
    mass = lambda i, j: area * (1.0 + (i == j)) / 12.0
    dot = lambda i, j: np.einsum("fi,fi->f", G[i], G[j])
    B = np.empty((P.shape[0], 3, 3))
    for a, (p, q) in enumerate(FACE_EDGES):
        for b, (r, s) in enumerate(FACE_EDGES):
            B[:, a, b] = (dot(q, s) * mass(p, r) - dot(q, r) * mass(p, s)
                          - dot(p, s) * mass(q, r) + dot(p, r) * mass(q, s))
    return B


def assemble_B(mesh, faces=None):
    """Boundary mass B over the mesh DOFs from the given triangles (default: the boundary
    of the unit cube). Edges without a DOF are skipped."""
    from .mesh import boundary_faces
    if faces is None:
        faces = boundary_faces(mesh.tets, mesh.n)
    Be = face_matrices(mesh.coords(faces))
    d = np.stack([mesh.dof_of_pairs(faces[:, a], faces[:, b]) for a, b in FACE_EDGES], axis=1)
    rows = np.repeat(d[:, :, None], 3, axis=2)
    cols = np.repeat(d[:, None, :], 3, axis=1)
    keep = (rows >= 0) & (cols >= 0)
    B = sp.coo_matrix((Be[keep], (rows[keep], cols[keep])), shape=(mesh.n_dof, mesh.n_dof)).tocsr()
    B.sum_duplicates()
    B.sort_indices()
    return B


def imp_sign(xi):
    """sign(xi) of Eq. imp with sign(0) = +1."""
    return -1.0 if xi < 0 else 1.0


def a_xi(K, M, k, xi, B=None):
    """A_xi = K - (k^2 + i xi) M (Eq. 2.2 with the real Whitney basis), minus
    i sign(xi) k B with the impedance condition (Eq. imp)."""
    A = K.astype(np.complex128) - (k * k + 1j * xi) * M.astype(np.complex128)
    if B is not None:
        A = A - 1j * imp_sign(xi) * k * B.astype(np.complex128)
    return A.tocsr()


def gauss_legendre01(q):
    """Gauss-Legendre nodes and weights on [0, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def duffy_rule(q=3):
    """Conical-product rule on the reference tetrahedron: (xi [Q, 3], weight [Q]).

    Weights sum to 1/6 (the reference volume)."""
    t, wt = gauss_legendre01(q)
    pts, wts = [], []
    for a in range(q):
        for b in range(q):
            for c in range(q):
                u, v, w = t[a], t[b], t[c]
                pts.append((u, (1 - u) * v, (1 - u) * (1 - v) * w))
                wts.append(wt[a] * wt[b] * wt[c] * (1 - u) ** 2 * (1 - v))
    return np.array(pts), np.array(wts)


def load_vector(mesh, F, q=3):
    """f_i = int F . w_i (Sec. 2.2; real basis so no conjugate), quadrature per tet.

    F: callable x [N, 3] -> complex [N, 3, R] (R right-hand sides) or [N, 3].
    Returns f [n_dof, R] (or [n_dof])."""
    P = tet_coords(mesh)
    G, vol = bary_gradients(P)
    xi, wq = duffy_rule(q)
    T = P.shape[0]
    f = None
    for qp in range(xi.shape[0]):
        lam = np.empty((T, 4))
        lam[:, 1:] = xi[qp]
        lam[:, 0] = 1.0 - xi[qp].sum()
        x = P[:, 0] + np.einsum("m,tmi->ti", xi[qp], P[:, 1:] - P[:, :1])
        Fx = F(x)
        squeeze = Fx.ndim == 2
        if squeeze:
            Fx = Fx[:, :, None]
        if f is None:
            f = np.zeros((mesh.n_dof, Fx.shape[2]), dtype=np.complex128)
        wgt = 6.0 * vol * wq[qp]
        for a, (p, r) in enumerate(LOCAL_EDGES):
            w = lam[:, p, None] * G[:, r] - lam[:, r, None] * G[:, p]  # [T, 3]
            contrib = np.einsum("ti,tir->tr", w, Fx) * wgt[:, None]
            dof = mesh.tet2dof[:, a]
            ok = dof >= 0
            np.add.at(f, dof[ok], contrib[ok])
    return f[:, 0] if squeeze else f


def bump_field(centres, pol, width):
    """F(x) = sum_b pol_b exp(-|x - c_b|^2 / width^2) for R right-hand sides.

    centres [R, B, 3], pol [R, B, 3] complex. Returns a callable for load_vector."""
    centres = np.asarray(centres, dtype=np.float64)
    pol = np.asarray(pol, dtype=np.complex128)

    def F(x):
        out = np.zeros((x.shape[0], 3, centres.shape[0]), dtype=np.complex128)
        for r in range(centres.shape[0]):
            for b in range(centres.shape[1]):
                d2 = np.sum((x - centres[r, b]) ** 2, axis=1)
                out[:, :, r] += np.exp(-d2 / width ** 2)[:, None] * pol[r, b][None, :]
        return out

    return F


def discrete_gradient(mesh):
    """G: interior edge x vertex incidence, (G phi)_e = phi(high) - phi(low)."""
    nv = (mesh.n + 1) ** 3
    r = np.repeat(np.arange(mesh.n_dof), 2)
    c = mesh.dof_edges.ravel()
    v = np.tile([-1.0, 1.0], mesh.n_dof)
    return sp.coo_matrix((v, (r, c)), shape=(mesh.n_dof, nv)).tocsr()


def interior_vertices(mesh):
    ijk = mesh.coords(np.arange((mesh.n + 1) ** 3)) * mesh.n
    return np.all((ijk > 0.5) & (ijk < mesh.n - 0.5), axis=1)

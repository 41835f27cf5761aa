"""Overlapping subdomains, coarse space and the additive Schwarz preconditioner.

Oracle (test infrastructure only).

Paper:
  * Sec. 3.1, Eq. 3.1: local spaces with zero tangential trace on the subdomain
    boundary; I^h(Omega_l) = DOFs whose edge lies in Omega_l; R^l selects them.
  * Sec. 3.2, Eq. 3.2: coarse restriction (R^0)_pj = psi_j^h(w_p^H).
  * Sec. 3.3, Eq. 3.3: A^l = R^l A (R^l)^T (minors for l >= 1; coarse Galerkin
    matrix for l = 0); Eq. 3.4: B^{-1} = sum_{l=0}^N (R^l)^T (A^l)^{-1} R^l.
    The one-level variant omits l = 0 (Sec. 6.2).
  * Sec. 6.1: overlapping subdomains are grown from a non-overlapping partition.

Readings:
  * subdomains are cube-aligned boxes: core boxes of `core` cells per axis
    (box i covers cells [core*i, min(core*(i+1), n))), each widened by `overlap`
    cells on every side and clipped to the unit cube. Local DOFs are the
    interior edges with both ends in the box and not lying on a box face
    (PEC on the subdomain boundary, Eq. 3.1). Subdomain id l = ix + N (iy + N iz).
  * coarse mesh: a Kuhn mesh with m cells per side, m dividing n, so it is nested
    in the fine mesh. psi_j(w) = int_{e_j} w . tau ds; w_p^H is linear on the coarse
    tetrahedron holding e_j, so the midpoint rule is exact:
    (R^0)_pj = w_p^H(midpoint_j) . (x_high - x_low).
  * local and coarse solves: sparse LU with partial pivoting (scipy SuperLU),
    like the paper's MUMPS direct solves (Sec. 6.1).
  * partition of unity for the restricted variants (Sec. 6.3): D^l is the 0/1 diagonal
    marking the DOFs that subdomain l owns, the owner being the core box that contains
    the edge midpoint (per axis cell index floor(mid / core), clipped to the last box).
    With overlap >= 1 the owner always holds the DOF, so sum_l (R^l)^T D^l R^l = I.
  * inexact coarse solve (Sec. 6.4): (A^0)^{-1} R^0 v is replaced by the result of an
    inner right-preconditioned GMRES on A^0 y = R^0 v -- unrestarted, y0 = 0, stopped at
    a relative Euclidean residual tol (the paper takes 1e-1) or after max_it iterations --
    preconditioned by a one-level Schwarz method on subdomains of the coarse mesh (boxes
    of the coarse mesh built by the same rules as on the fine mesh). The paper's inner
    preconditioner is the one-level ImpRAS (impedance conditions on the subdomain
    boundaries); here the subdomain problems keep the PEC conditions of Eq. 3.1 (one-level
    RAS or AS).
  * impedance problems (Eq. imp, mesh bc "imp"): the local problems are those of ImpRAS
    (Sec. 6.3): the Maxwell problem on the box with the impedance condition on its whole
    boundary -- on the part inside the domain by the definition of ImpRAS, on the part on
    the domain boundary because the global problem has it there. The local DOFs are then all
    edges of the closed box (its faces included), and A^l is the Galerkin matrix of the box:
    element matrices of the tetrahedra inside the box, minus i sign(xi) k times the
    tangential mass of the box-surface triangles (not a minor of A). The additive, restricted
    and hybrid forms are built from these local solves as before (ImpAS, ImpRAS, ImpHRAS,
    ADEF1-ImpRAS); the coarse problem is the impedance problem on the coarse mesh.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import KuhnMesh, vertex_ijk, boundary_faces, DIRS, LOCAL_EDGES
from . import fem


def subdomain_boxes(n, core, overlap):
    """List of vertex-index boxes (lo[3], hi[3]) in subdomain order."""
    N = -(-n // core)
    spans = []
    for i in range(N):
        lo = max(core * i - overlap, 0)
        hi = min(min(core * (i + 1), n) + overlap, n)
        spans.append((lo, hi))
    boxes = []
    for iz in range(N):
        for iy in range(N):
            for ix in range(N):
                boxes.append((np.array([spans[ix][0], spans[iy][0], spans[iz][0]]),
                              np.array([spans[ix][1], spans[iy][1], spans[iz][1]])))
    return boxes


def local_dofs(mesh, lo, hi, closed=False):
    """Sorted global DOFs of the box [lo, hi] (vertex indices), Eq. 3.1 reading; closed:
    the edges on the box faces included (impedance local problems)."""
    a = vertex_ijk(mesh.dof_edges[:, 0], mesh.n)
    b = vertex_ijk(mesh.dof_edges[:, 1], mesh.n)
    inside = np.all((a >= lo) & (a <= hi) & (b >= lo) & (b <= hi), axis=1)
    if closed:
        return np.nonzero(inside)[0]
    on_face = np.zeros_like(inside)
    for ax in range(3):
        for val in (lo[ax], hi[ax]):
            on_face |= (a[:, ax] == val) & (b[:, ax] == val)
    return np.nonzero(inside & ~on_face)[0]


def restriction(idx, n_dof):
    """R^l as a sparse 0/1 matrix (Eq. 3.1)."""
    return sp.csr_matrix((np.ones(len(idx)), (np.arange(len(idx)), idx)),
                         shape=(len(idx), n_dof))


def coarse_restriction(fine: KuhnMesh, coarse: KuhnMesh):
    """R^0 [n_c, n] of Eq. 3.2 on nested Kuhn meshes (midpoint rule, exact)."""
    n, m = fine.n, coarse.n
    assert n % m == 0, "coarse mesh must be nested (m divides n)"
    H = 1.0 / m
    xa = fine.coords(fine.dof_edges[:, 0])
    xb = fine.coords(fine.dof_edges[:, 1])
    mid = 0.5 * (xa + xb)
    t = xb - xa
    s = mid / H
    cube = np.clip(np.floor(s).astype(np.int64), 0, m - 1)
    loc = s - cube
    # Kuhn simplex of the coarse cube holding the midpoint: local coordinates in
    # decreasing order give its vertex path (ties: any containing simplex).
    perm = np.argsort(-loc, axis=1, kind="stable")
    eye = np.eye(3, dtype=np.int64)
    path = [cube]
    for k in range(3):
        path.append(path[-1] + eye[perm[:, k]])
    path = np.stack(path, axis=1)  # [n, 4, 3] coarse grid indices
    P = path * H
    G, _ = fem.bary_gradients(P)  # [n, 4, 3]
    Mx = np.ones((fine.n_dof, 4, 4))
    Mx[:, :, 1:] = P
    rhs = np.concatenate([np.ones((fine.n_dof, 1)), mid], axis=1)
    lam = np.linalg.solve(np.transpose(Mx, (0, 2, 1)), rhs[:, :, None])[:, :, 0]
    vid = path[:, :, 0] + (m + 1) * (path[:, :, 1] + (m + 1) * path[:, :, 2])
    lut = np.full(7 * (m + 1) ** 3, -1, dtype=np.int64)
    lut[coarse.dof_key] = np.arange(coarse.n_dof)
    rows, cols, vals = [], [], []
    for (p, q) in LOCAL_EDGES:
        lo, hi = vid[:, p], vid[:, q]
        dvec = vertex_ijk(hi, m) - vertex_ijk(lo, m)
        dirs = np.full(fine.n_dof, -1, dtype=np.int64)
        for k, dv in enumerate(DIRS):
            dirs[np.all(dvec == dv, axis=1)] = k
        assert np.all(dirs >= 0)
        dof = lut[7 * lo + dirs]
        w = lam[:, p, None] * G[:, q] - lam[:, q, None] * G[:, p]
        val = np.einsum("ji,ji->j", w, t)
        keep = (dof >= 0) & (val != 0.0)
        rows.append(dof[keep])
        cols.append(np.nonzero(keep)[0])
        vals.append(val[keep])
    R0 = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(coarse.n_dof, fine.n_dof)).tocsr()
    R0.sum_duplicates()
    return R0


class Schwarz:
    """One- or two-level additive Schwarz preconditioner of Eq. 3.4."""

    def __init__(self, mesh, A_prec, core, overlap, coarse_m=0, k=None, xi_prec=None):
        self.mesh = mesh
        self.imp = getattr(mesh, "bc", "pec") == "imp"
        self.k, self.xi_prec = k, xi_prec
        self.core, self.overlap = core, overlap
        self.boxes = subdomain_boxes(mesh.n, core, overlap)
        self.idx = [local_dofs(mesh, lo, hi, closed=self.imp) for lo, hi in self.boxes]
        self.A_prec = A_prec.tocsr()
        self.lus = None
        self.coarse = None
        self.inner = None  # one-level Schwarz on the coarse mesh (inexact coarse solve)
        if coarse_m:
            cm = KuhnMesh(coarse_m, "imp" if self.imp else "pec")
            Kc, Mc = fem.assemble_KM(cm)
            self.coarse_mesh = cm
            self.R0 = coarse_restriction(mesh, cm)
            # Galerkin matrix on Q_H (Eq. 3.3, l = 0), with the boundary term when impedance
            self.A0 = fem.a_xi(Kc, Mc, k, xi_prec, fem.assemble_B(cm) if self.imp else None)

    def owner(self):
        """Owning subdomain of every DOF: the core box holding the edge midpoint."""
        n, core = self.mesh.n, self.core
        N = -(-n // core)
        a = vertex_ijk(self.mesh.dof_edges[:, 0], n)
        b = vertex_ijk(self.mesh.dof_edges[:, 1], n)
        mid2 = a + b  # twice the midpoint, in vertex units
        box = np.minimum(mid2 // (2 * core), N - 1)
        return box[:, 0] + N * (box[:, 1] + N * box[:, 2])

    def partition_of_unity(self):
        """D^l of Sec. 6.3 as boolean masks over the local DOFs of every subdomain."""
        own = self.owner()
        return [own[i] == l for l, i in enumerate(self.idx)]

    def minor(self, l):
        """A^l = R^l A (R^l)^T (Eq. 3.3) as a sparse matrix; for impedance problems the
        Galerkin matrix of the box with the impedance condition on its boundary."""
        i = self.idx[l]
        if self.imp:
            return self.box_matrix(l)
        return self.A_prec[i][:, i]

    def box_matrix(self, l):
        """ImpRAS local matrix (Sec. 6.3): K - (k^2 + i xi) M - i sign(xi) k B assembled over
        the tetrahedra inside box l and the triangles on its surface, on its closed-box DOFs."""
        mesh, (lo, hi) = self.mesh, self.boxes[l]
        idx = self.idx[l]
        ijk = vertex_ijk(mesh.tets, mesh.n)
        inside = np.all((ijk >= lo) & (ijk <= hi), axis=(1, 2))
        tets = mesh.tets[inside]
        Ke, Me = fem.element_matrices(mesh.coords(tets))
        d = np.searchsorted(idx, mesh.tet2dof[inside])
        nl = len(idx)
        rows = np.repeat(d[:, :, None], 6, axis=2).ravel()
        cols = np.repeat(d[:, None, :], 6, axis=1).ravel()
        K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(nl, nl)).tocsr()
        M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(nl, nl)).tocsr()
        faces = boundary_faces(tets, mesh.n, tuple(lo), tuple(hi))
        Be = fem.face_matrices(mesh.coords(faces))
        fd = np.stack([np.searchsorted(idx, mesh.dof_of_pairs(faces[:, a], faces[:, b]))
                       for a, b in fem.FACE_EDGES], axis=1)
        B = sp.coo_matrix((Be.ravel(), (np.repeat(fd[:, :, None], 3, axis=2).ravel(),
                                        np.repeat(fd[:, None, :], 3, axis=1).ravel())), shape=(nl, nl)).tocsr()
        return fem.a_xi(K, M, self.k, self.xi_prec, B)

    def set_inner_coarse(self, core, overlap, tol=0.1, max_it=100, kind="ras"):
        """Solve the coarse problem inexactly by inner GMRES (Sec. 6.4), preconditioned by
        one-level Schwarz (kind "as" or "ras") on boxes of `core` coarse cells widened by
        `overlap` coarse cells."""
        if not hasattr(self, "A0"):
            raise ValueError("no coarse level")
        self.inner = Schwarz(self.coarse_mesh, self.A0, core, overlap, k=self.k, xi_prec=self.xi_prec)
        self.inner_tol, self.inner_max_it, self.inner_kind = tol, max_it, kind
        self.inner_its = []  # inner iterations of every coarse solve, in order

    def factor(self, subset=None):
        ls = range(len(self.idx)) if subset is None else subset
        self.lus = {l: spla.splu(self.minor(l).tocsc()) for l in ls}
        if self.inner is not None:
            self.inner.factor()
        elif hasattr(self, "A0"):
            self.coarse = spla.splu(self.A0.tocsc())

    def local_solve(self, l, r_l):
        return self.lus[l].solve(r_l)

    def coarse_solve(self, rc):
        """(A^0)^{-1} rc: direct, or the inner GMRES of Sec. 6.4 when set."""
        if self.inner is None:
            return self.coarse.solve(rc)
        if rc.ndim == 2:  # one inner solve per column
            return np.stack([self.coarse_solve(rc[:, q]) for q in range(rc.shape[1])], axis=1)
        from .gmres import gmres
        A0, inner, kind = self.A0, self.inner, self.inner_kind
        y, its, _, _ = gmres(lambda u: A0 @ u, lambda u: inner.apply(u, levels=(1,), kind=kind), rc,
                             self.inner_tol, 0, self.inner_max_it)
        self.inner_its.append(its)
        return y

    def coarse_correction(self, v):
        """G v with G = (R^0)^T (A^0)^{-1} R^0 (the coarse term of Eq. 3.4)."""
        return self.R0.T @ self.coarse_solve(self.R0 @ v)

    def ras1(self, v):
        """One-level restricted additive Schwarz: sum_l (R^l)^T D^l (A^l)^{-1} R^l v (Sec. 6.3)."""
        if not hasattr(self, "_pou"):
            self._pou = self.partition_of_unity()
        z = np.zeros_like(v, dtype=np.complex128)
        for l, i in enumerate(self.idx):
            zl = self.local_solve(l, v[i])
            d = self._pou[l]
            z[i[d]] += zl[d]
        return z

    def apply(self, v, levels=(1, 0), kind="as"):
        """Preconditioner application, v [n] or [n, R].

        kind "as": sum_l (R^l)^T (A^l)^{-1} R^l v over the levels given (Eq. 3.4);
        "ras": the restricted local sum plus the coarse term if level 0 is given (Eq. RAS2);
        "hras": (I - G A) B_RAS1^{-1} (I - A G) + G (Eq. HRAS);
        "adef1": B_RAS1^{-1} (I - A G) + G (Eq. ADEF1ras); A = A_{xi_prec}."""
        if kind in ("hras", "adef1"):
            A = self.A_prec
            gv = self.coarse_correction(v)
            u = self.ras1(v - A @ gv)
            if kind == "adef1":
                return u + gv
            return u - self.coarse_correction(A @ u) + gv
        z = np.zeros_like(v, dtype=np.complex128)
        if 1 in levels:
            if kind == "ras":
                z += self.ras1(v)
            else:
                for l, i in enumerate(self.idx):
                    z[i] += self.local_solve(l, v[i])
        if 0 in levels and (self.coarse is not None or self.inner is not None):
            z += self.coarse_correction(v)
        return z

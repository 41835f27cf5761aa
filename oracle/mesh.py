"""Uniform Kuhn tetrahedral mesh of the unit cube and lowest-order edge DOFs.

Oracle (test infrastructure only).

Paper: Sec. 2.2 (conforming tetrahedral mesh, Nedelec space Q_h whose tangential
trace vanishes on the boundary, Eq. 1.4 PEC condition); DOFs of the lowest order
space are the edges of the mesh.

Readings where the paper is silent (it used FreeFem++ meshes):
  * mesh: n^3 cubes of side h = 1/n, each split into 6 Kuhn tetrahedra. The tetrahedron
    of cube c and permutation s = (s0, s1, s2) has the vertex path
    c, c + e_s0, c + e_s0 + e_s1, c + (1, 1, 1). Permutations are taken in lexicographic
    order; tet id = 6 * cube id + permutation index, cube id = i + n (j + n l).
  * vertex id v(i, j, l) = i + (n+1)(j + (n+1) l).
  * edges are oriented from the lower to the higher vertex id.
  * an edge is a PEC (boundary) edge when both endpoints lie on one boundary face;
    those DOFs are removed.
  * DOF numbering: interior edges sorted by key 7 * v_low + d, d the index of
    v_high - v_low in DIRS.
  * impedance boundary condition (Eq. imp, bc="imp"): the condition is natural, so every
    edge of the mesh carries a DOF (same key order); the boundary enters the matrix
    through the boundary triangles (fem.assemble_B).

This module derives everything from the tetrahedra by brute force (unique vertex
pairs), not from a per-vertex enumeration.
"""
import itertools

import numpy as np

DIRS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]],
                dtype=np.int64)
PERMS = list(itertools.permutations(range(3)))  # lexicographic
LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def vertex_ijk(v, n):
    """Integer grid coordinates of vertex ids v (array) on the n-cell mesh."""
    v = np.asarray(v, dtype=np.int64)
    i = v % (n + 1)
    j = (v // (n + 1)) % (n + 1)
    l = v // ((n + 1) * (n + 1))
    return np.stack([i, j, l], axis=-1)


def vertex_id(ijk, n):
    ijk = np.asarray(ijk, dtype=np.int64)
    return ijk[..., 0] + (n + 1) * (ijk[..., 1] + (n + 1) * ijk[..., 2])


def kuhn_tets(n):
    """Tetrahedra [6 n^3, 4] as path-ordered vertex ids (increasing)."""
    cubes = np.array([(i, j, l) for l in range(n) for j in range(n) for i in range(n)],
                     dtype=np.int64).reshape(-1, 3)
    tets = np.empty((cubes.shape[0], 6, 4), dtype=np.int64)
    eye = np.eye(3, dtype=np.int64)
    for p, s in enumerate(PERMS):
        c0 = cubes
        c1 = c0 + eye[s[0]]
        c2 = c1 + eye[s[1]]
        c3 = c2 + eye[s[2]]
        for k, c in enumerate((c0, c1, c2, c3)):
            tets[:, p, k] = vertex_id(c, n)
    return tets.reshape(-1, 4)


def all_edges(tets):
    """Unique edges [E, 2] (low, high vertex id) of the given tetrahedra, sorted."""
    pairs = []
    for a, b in LOCAL_EDGES:
        pairs.append(np.stack([np.minimum(tets[:, a], tets[:, b]),
                               np.maximum(tets[:, a], tets[:, b])], axis=1))
    pairs = np.concatenate(pairs)
    return np.unique(pairs, axis=0)


def edge_dir(pairs, n):
    """Direction index in DIRS of each oriented edge (low -> high)."""
    d = vertex_ijk(pairs[:, 1], n) - vertex_ijk(pairs[:, 0], n)
    out = np.full(pairs.shape[0], -1, dtype=np.int64)
    for k, dv in enumerate(DIRS):
        out[np.all(d == dv, axis=1)] = k
    assert np.all(out >= 0), "edge with a direction outside the Kuhn set"
    return out


def is_pec_edge(pairs, n):
    """True where both endpoints lie on one face of the unit cube (Eq. 1.4)."""
    a = vertex_ijk(pairs[:, 0], n)
    b = vertex_ijk(pairs[:, 1], n)
    on = np.zeros(pairs.shape[0], dtype=bool)
    for ax in range(3):
        for val in (0, n):
            on |= (a[:, ax] == val) & (b[:, ax] == val)
    return on


class KuhnMesh:
    """Mesh, edges and DOF numbering for n cells per side; bc "pec" (Eq. 1.4: boundary
    edges carry no DOF) or "imp" (Eq. imp: every edge is a DOF)."""

    def __init__(self, n, bc="pec"):
        if bc not in ("pec", "imp"):
            raise ValueError(bc)
        self.n = int(n)
        self.h = 1.0 / n
        self.bc = bc
        self.tets = kuhn_tets(n)
        self.edges = all_edges(self.tets)  # [E, 2], sorted by (low, high)
        self.edge_dir = edge_dir(self.edges, n)
        self.key = 7 * self.edges[:, 0] + self.edge_dir
        interior = ~is_pec_edge(self.edges, n) if bc == "pec" else np.ones(self.edges.shape[0], dtype=bool)
        order = np.argsort(self.key[interior], kind="stable")
        self.dof_edges = self.edges[interior][order]  # [n_dof, 2]
        self.dof_key = self.key[interior][order]
        self.dof_dir = self.edge_dir[interior][order]
        self.n_dof = self.dof_edges.shape[0]
        # map every key to its DOF (-1 for PEC edges)
        self._key_to_dof = {int(k): i for i, k in enumerate(self.dof_key)}
        self.tet2dof = self._tet_dofs()

    def coords(self, v):
        return vertex_ijk(v, self.n) * self.h

    def dof_of_pairs(self, lo, hi):
        """DOF index of oriented edges (lo < hi), -1 when the edge is PEC."""
        pairs = np.stack([lo, hi], axis=1)
        keys = 7 * lo + edge_dir(pairs, self.n)
        return np.array([self._key_to_dof.get(int(k), -1) for k in keys], dtype=np.int64)

    def _tet_dofs(self):
        out = np.empty((self.tets.shape[0], 6), dtype=np.int64)
        lut = np.full(7 * (self.n + 1) ** 3, -1, dtype=np.int64)
        lut[self.dof_key] = np.arange(self.n_dof)
        for k, (a, b) in enumerate(LOCAL_EDGES):
            lo, hi = self.tets[:, a], self.tets[:, b]
            assert np.all(lo < hi)
            pairs = np.stack([lo, hi], axis=1)
            out[:, k] = lut[7 * lo + edge_dir(pairs, self.n)]
        return out


def boundary_faces(tets, n, lo=(0, 0, 0), hi=None):
    """Triangles of the given tetrahedra lying on a face of the box [lo, hi] (vertex
    indices; default the unit cube): [F, 3] vertex ids in increasing order. Found by brute
    force: a tetrahedron face whose three vertices share a coordinate equal to a box bound."""
    hi = (n, n, n) if hi is None else hi
    out = []
    for t in tets:
        for drop in range(4):
            f = np.sort(np.delete(t, drop))
            ijk = vertex_ijk(f, n)
            for ax in range(3):
                col = ijk[:, ax]
                if np.all(col == col[0]) and col[0] in (lo[ax], hi[ax]):
                    out.append(f)
                    break
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def count_closed_box_edges(a, b, c):
    """Closed form for all edges of an a x b x c Kuhn box (its faces included): per
    direction D the number of start vertices, prod over axes of (len + 1 - D)."""
    L = (a, b, c)
    return int(sum(np.prod([L[ax] + 1 - D[ax] for ax in range(3)]) for D in DIRS))


def count_all_edges(n):
    """Closed form 3n(n+1)^2 + 3n^2(n+1) + n^3 (axis, face-diagonal, body-diagonal)."""
    return 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3


def count_interior_edges(a, b=None, c=None):
    """Closed form for the edges of an a x b x c Kuhn box not lying on its faces."""
    if b is None:
        b = c = a
    return (a * (b - 1) * (c - 1) + b * (a - 1) * (c - 1) + c * (a - 1) * (b - 1)
            + a * b * (c - 1) + a * c * (b - 1) + b * c * (a - 1) + a * b * c)

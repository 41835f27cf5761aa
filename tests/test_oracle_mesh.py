"""Pins for oracle.mesh: closed-form counts, Euler's formula, conformity and an
independent second derivation of the edge set and of the PEC classification."""
import itertools

import numpy as np
import pytest

from oracle.mesh import (KuhnMesh, DIRS, count_all_edges, count_interior_edges,
                         vertex_ijk, vertex_id)
from oracle import fem


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_counts_closed_form(n):
    m = KuhnMesh(n)
    assert m.tets.shape[0] == 6 * n ** 3
    assert m.edges.shape[0] == count_all_edges(n)
    assert m.n_dof == count_interior_edges(n)


def test_counts_table():
    # 10 cells: 7,930 edges, 6,130 PEC-interior DOFs; 12 cells: 13,428 / 10,836
    assert count_all_edges(10) == 7930 and count_interior_edges(10) == 6130
    assert count_all_edges(12) == 13428 and count_interior_edges(12) == 10836
    assert count_interior_edges(7) == 1981 and count_interior_edges(6) == 1206
    assert count_interior_edges(40) == 433720 and count_interior_edges(60) == 1479780


@pytest.mark.parametrize("n", [1, 2, 3])
def test_euler_and_conformity(n):
    m = KuhnMesh(n)
    faces = {}
    for t in m.tets:
        for f in itertools.combinations(sorted(int(x) for x in t), 3):
            faces[f] = faces.get(f, 0) + 1
    V = (n + 1) ** 3
    # Euler characteristic of a ball: V - E + F - T = 1
    assert V - m.edges.shape[0] + len(faces) - m.tets.shape[0] == 1
    # conforming: every face shared by two tets, except the 12 n^2 boundary triangles
    counts = np.array(list(faces.values()))
    assert set(counts.tolist()) <= {1, 2}
    assert int(np.sum(counts == 1)) == 12 * n * n


@pytest.mark.parametrize("n", [1, 2, 4])
def test_tet_volumes(n):
    m = KuhnMesh(n)
    _, vol = fem.bary_gradients(m.coords(m.tets))
    assert np.allclose(vol, 1.0 / (6 * n ** 3), rtol=1e-13)
    assert abs(vol.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_edges_from_direction_enumeration(n):
    """Edges from tets == edges (v, v + d) over the 7 Kuhn directions inside the grid."""
    m = KuhnMesh(n)
    pairs = set()
    for v in range((n + 1) ** 3):
        ijk = vertex_ijk(v, n)
        for d in DIRS:
            w = ijk + d
            if np.all(w <= n):
                pairs.add((v, int(vertex_id(w, n))))
    assert pairs == set(map(tuple, m.edges.tolist()))


@pytest.mark.parametrize("n", [2, 3, 4])
def test_pec_by_midpoint(n):
    """An edge lies on the boundary iff its midpoint does (convex domain)."""
    m = KuhnMesh(n)
    mid = 0.5 * (m.coords(m.edges[:, 0]) + m.coords(m.edges[:, 1]))
    on = np.any((np.abs(mid) < 1e-12) | (np.abs(mid - 1) < 1e-12), axis=1)
    interior = set(map(tuple, m.edges[~on].tolist()))
    assert interior == set(map(tuple, m.dof_edges.tolist()))
    # numbering is increasing in the key 7 v_low + d
    assert np.all(np.diff(m.dof_key) > 0)


def test_tet_paths_monotone():
    m = KuhnMesh(3)
    d = np.diff(m.tets, axis=1)
    assert np.all(d > 0)
    # every tet contains the main diagonal of its cube
    ijk0 = vertex_ijk(m.tets[:, 0], 3)
    ijk3 = vertex_ijk(m.tets[:, 3], 3)
    assert np.all(ijk3 - ijk0 == 1)


def test_numbering_conventions_by_hand():
    """The documented numbering, checked on hand-computed cases. DOFs are sorted by the key
    7 v_low + d, with d indexing the directions (1,0,0), (0,1,0), (0,0,1), (1,1,0), (1,0,1),
    (0,1,1), (1,1,1). On the single cube with all edges (n = 1, impedance), vertex 0 = (0,0,0)
    starts one edge in every direction, to the vertices 1, 2, 4, 3, 5, 6, 7 (vertex id
    i + 2 (j + 2 l)). Columns of tet2dof follow the local edges 01, 02, 03, 12, 13, 23."""
    m = KuhnMesh(1, "imp")
    assert m.n_dof == 19
    first = [tuple(e) for e in m.dof_edges[:7].tolist()]
    assert first == [(0, 1), (0, 2), (0, 4), (0, 3), (0, 5), (0, 6), (0, 7)]
    assert m.dof_key[:7].tolist() == list(range(7))
    # the tetrahedron of permutation (0, 1, 2): path 0 -> 1 -> 3 -> 7
    assert m.tets[0].tolist() == [0, 1, 3, 7]
    d = {tuple(e): i for i, e in enumerate(m.dof_edges.tolist())}
    assert m.tet2dof[0].tolist() == [d[(0, 1)], d[(0, 3)], d[(0, 7)], d[(1, 3)], d[(1, 7)], d[(3, 7)]]
    for t in (m, KuhnMesh(3)):
        for k, (p, q) in enumerate([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]):
            assert np.array_equal(t.tet2dof[:, k], t.dof_of_pairs(t.tets[:, p], t.tets[:, q]))

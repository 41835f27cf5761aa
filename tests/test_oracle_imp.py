"""Pins for the impedance problem (Eq. imp) and the ImpRAS local problems (Sec. 6.3) in the
oracle: DOF and boundary-triangle counts (closed forms), the tangential boundary mass
against an independent quadrature of the projected three-dimensional Whitney functions,
the boundary form of discrete gradients of linear functions (exact), the structure of B,
the box matrices against a standalone impedance mesh of the box, a single subdomain giving
the exact inverse, nested coarse Galerkin, sign(-xi) conjugation, and GMRES with the
impedance preconditioners against a direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.mesh import (KuhnMesh, boundary_faces, count_all_edges, count_closed_box_edges, is_pec_edge,
                         vertex_ijk, LOCAL_EDGES)
from oracle import fem, dd
from oracle.problem import Problem


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_counts(n):
    m = KuhnMesh(n, "imp")
    assert m.n_dof == count_all_edges(n) == m.edges.shape[0]
    f = boundary_faces(m.tets, n)
    assert len(f) == 12 * n * n  # 6 faces x n^2 squares x 2 triangles
    P = m.coords(f)
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    assert abs(area.sum() - 6.0) < 1e-12


@pytest.mark.parametrize("n,core,overlap", [(9, 3, 1), (10, 4, 1), (6, 3, 0)])
def test_closed_box_counts(n, core, overlap):
    m = KuhnMesh(n, "imp")
    for lo, hi in dd.subdomain_boxes(n, core, overlap):
        idx = dd.local_dofs(m, lo, hi, closed=True)
        assert len(idx) == count_closed_box_edges(*(hi - lo).tolist())


def _quad_face_mass(m, faces):
    """int_F (w_a)_T . (w_b)_T by the 3-point edge-midpoint rule (exact for quadratics),
    with w from the barycentrics of a tetrahedron holding the face, projected on the
    face plane. Independent of the surface-gradient route of fem.face_matrices."""
    out = np.zeros((len(faces), 3, 3))
    tets = m.tets
    for fi, f in enumerate(faces):
        t = next(t for t in tets if set(f) <= set(t))
        P = m.coords(t)
        G, vol = fem.bary_gradients(P[None])
        G = G[0]
        X = m.coords(f)
        nrm = np.cross(X[1] - X[0], X[2] - X[0])
        area = 0.5 * np.linalg.norm(nrm)
        nrm /= np.linalg.norm(nrm)
        Mx = np.ones((4, 4))
        Mx[:, 1:] = P
        pos = {int(v): i for i, v in enumerate(t)}
        pts = [0.5 * (X[0] + X[1]), 0.5 * (X[0] + X[2]), 0.5 * (X[1] + X[2])]
        for x in pts:
            lam = np.linalg.solve(Mx.T, np.concatenate([[1.0], x]))
            ws = []
            for a, b in fem.FACE_EDGES:
                p, q = pos[int(f[a])], pos[int(f[b])]
                w = lam[p] * G[q] - lam[q] * G[p]
                ws.append(w - np.dot(w, nrm) * nrm)
            for i in range(3):
                for j in range(3):
                    out[fi, i, j] += area / 3.0 * np.dot(ws[i], ws[j])
    return out


def test_face_mass_against_quadrature():
    m = KuhnMesh(3, "imp")
    f = boundary_faces(m.tets, 3)[::7]
    B = fem.face_matrices(m.coords(f))
    Q = _quad_face_mass(m, f)
    assert np.allclose(B, Q, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("coef,expect", [((1, 0, 0), 4.0), ((1, 2, 3), 56.0), ((0, 0, 2), 16.0)])
def test_boundary_form_of_linear_gradients(coef, expect):
    """phi linear: the interpolant is exact, G phi the exact edge DOFs of grad phi, and
    (G phi)^T B (G phi) = int_{boundary} |grad_T phi|^2 (faces of unit area); K G phi = 0."""
    n = 4
    m = KuhnMesh(n, "imp")
    K, M = fem.assemble_KM(m)
    B = fem.assemble_B(m)
    X = m.coords(np.arange((n + 1) ** 3))
    phi = X @ np.array(coef, dtype=float)
    g = fem.discrete_gradient(m) @ phi
    assert abs(g @ (B @ g) - expect) < 1e-11
    assert np.abs(K @ g).max() < 1e-10
    assert abs(g @ (M @ g) - float(np.dot(coef, coef))) < 1e-11


def test_B_structure_and_interior_gradients():
    n = 4
    m = KuhnMesh(n, "imp")
    B = fem.assemble_B(m)
    assert abs(B - B.T).max() == 0.0
    ev = np.linalg.eigvalsh(B.toarray())
    assert ev.min() > -1e-13
    bnd = is_pec_edge(m.dof_edges, n)
    rows, cols = B.nonzero()
    assert np.all(bnd[rows] & bnd[cols])
    # grad phi with phi = 0 on the boundary has no tangential trace
    rng = np.random.default_rng(2)
    ijk = vertex_ijk(np.arange((n + 1) ** 3), n)
    inner = np.all((ijk > 0) & (ijk < n), axis=1)
    phi = np.where(inner, rng.standard_normal((n + 1) ** 3), 0.0)
    assert np.abs(B @ (fem.discrete_gradient(m) @ phi)).max() < 1e-13


def test_box_matrix_is_standalone_impedance_matrix():
    """The ImpRAS matrix of an interior box is the impedance Galerkin matrix of a separate
    Kuhn mesh of the box (K scales like 1/h, M like h, B not at all)."""
    n, k, xi = 9, 3.0, 2.0
    m = KuhnMesh(n, "imp")
    K, M = fem.assemble_KM(m)
    S = dd.Schwarz(m, fem.a_xi(K, M, k, xi, fem.assemble_B(m)), 3, 0, k=k, xi_prec=xi)
    l = 13  # the centre box [3, 6]^3
    lo, hi = S.boxes[l]
    assert np.all(lo == 3) and np.all(hi == 6)
    mb = KuhnMesh(3, "imp")
    Kb, Mb = fem.assemble_KM(mb)
    s = mb.h / m.h
    Ab = fem.a_xi(Kb * s, Mb / s, k, xi, fem.assemble_B(mb))
    Al = S.box_matrix(l)
    assert abs(Al - Ab).max() < 1e-12 * abs(Ab).max()


def test_single_subdomain_is_exact():
    n, k = 4, 2.0
    P = Problem(n, k, 4.0, 4.0, n, 0, bc="imp")
    P.factor()
    assert abs(P.dd.box_matrix(0) - P.A_prec).max() < 1e-13
    rng = np.random.default_rng(1)
    b = rng.standard_normal(P.n_dof) + 1j * rng.standard_normal(P.n_dof)
    x, st = P.solve(b, tol=1e-12)
    assert st[0][0] == 1 and st[0][2]


def test_nested_coarse_galerkin_with_boundary_term():
    n, m_, k, xi = 6, 3, 2.5, 1.5
    f = KuhnMesh(n, "imp")
    K, M = fem.assemble_KM(f)
    A = fem.a_xi(K, M, k, xi, fem.assemble_B(f))
    S = dd.Schwarz(f, A, 3, 1, coarse_m=m_, k=k, xi_prec=xi)
    G = S.R0 @ A @ S.R0.T
    assert abs(G - S.A0).max() < 1e-12 * abs(S.A0).max()


def test_negative_xi_conjugates():
    m = KuhnMesh(3, "imp")
    K, M = fem.assemble_KM(m)
    B = fem.assemble_B(m)
    assert abs(fem.a_xi(K, M, 2.0, -3.0, B) - fem.a_xi(K, M, 2.0, 3.0, B).conj()).max() == 0.0
    # xi = 0 takes sign +1: the impedance term is -i k B
    A0 = fem.a_xi(K, M, 2.0, 0.0, B)
    assert abs(A0 - (K - 4.0 * M - 2.0j * B)).max() < 1e-14


@pytest.mark.parametrize("kind", ["as", "ras", "hras", "adef1"])
def test_impedance_gmres_matches_direct(kind):
    P = Problem(6, 3.0, 0.0, 3.0, 3, 1, coarse_m=3, kind=kind, bc="imp")
    P.factor()
    rng = np.random.default_rng(4)
    b = rng.standard_normal(P.n_dof) + 1j * rng.standard_normal(P.n_dof)
    x, st = P.solve(b, tol=1e-10, max_it=300)
    assert st[0][2]
    xd = spla.spsolve(P.A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)

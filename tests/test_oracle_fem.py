"""Pins for oracle.fem: element matrices against an independent evaluation of the
Whitney basis definition, exact reproduction of constant and rotational fields,
the discrete-gradient kernel of curl curl, complex symmetry, the quadrature rule,
first-order convergence to two manufactured solutions (a divergence-free field and a
gradient), and second-order closeness of the discrete solution to the edge interpolant."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.mesh import KuhnMesh, LOCAL_EDGES
from oracle import fem


def _bary_by_volumes(P, x):
    """Barycentric coordinates of x in tet P from signed sub-volume ratios."""
    def vol(a, b, c, d):
        return np.linalg.det(np.stack([b - a, c - a, d - a])) / 6.0
    V = vol(*P)
    lam = []
    for i in range(4):
        Q = [P[j] if j != i else x for j in range(4)]
        lam.append(vol(*Q) / V)
    return np.array(lam)


def _whitney(P, x, p, q, eps=0.25):
    """w_pq(x) = lam_p grad lam_q - lam_q grad lam_p, gradients by central differences
    (exact for affine functions at any step, up to rounding)."""
    lam = _bary_by_volumes(P, x)
    grad = np.zeros((4, 3))
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = eps
        grad[:, ax] = (_bary_by_volumes(P, x + e) - _bary_by_volumes(P, x - e)) / (2 * eps)
    return lam[p] * grad[q] - lam[q] * grad[p]


def _curl_whitney(P, p, q, eps=0.25):
    x0 = P.mean(axis=0)
    J = np.zeros((3, 3))
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = eps
        J[:, ax] = (_whitney(P, x0 + e, p, q) - _whitney(P, x0 - e, p, q)) / (2 * eps)
    return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])


TETS = [np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float),
        np.array([[0.1, 0.2, 0.0], [1.3, 0.1, 0.2], [0.2, 0.9, 0.1], [0.3, 0.2, 1.1]]),
        np.array([[0, 0, 0], [0.25, 0, 0], [0.25, 0.25, 0], [0.25, 0.25, 0.25]])]


@pytest.mark.parametrize("P", TETS)
def test_element_matrices_vs_definition(P):
    Ke, Me = fem.element_matrices(P[None])
    # independent quadrature: a degree-2 exact rule built from a different q
    xi, wq = fem.duffy_rule(4)
    vol = abs(np.linalg.det(P[1:] - P[0])) / 6.0
    Mq = np.zeros((6, 6))
    for qp in range(xi.shape[0]):
        x = P[0] + xi[qp] @ (P[1:] - P[0])
        W = np.array([_whitney(P, x, p, q) for p, q in LOCAL_EDGES])
        Mq += 6 * vol * wq[qp] * W @ W.T
    C = np.array([_curl_whitney(P, p, q) for p, q in LOCAL_EDGES])
    Kq = vol * C @ C.T
    assert np.allclose(Me[0], Mq, rtol=1e-12, atol=1e-13 * np.abs(Mq).max())
    assert np.allclose(Ke[0], Kq, rtol=1e-12, atol=1e-13 * np.abs(Kq).max())


def test_reference_tet_closed_form():
    """Reference tet: grad lam = (-1,-1,-1), e1, e2, e3 and |T| = 1/6. For the edge
    (0,1), int |lam0 e1 - lam1 grad lam0|^2 = |T| [2/20 * 1 - 2 * 1/20 * (-1) + 2/20 * 3]
    = 1/12 by hand."""
    Ke, Me = fem.element_matrices(TETS[0][None])
    assert abs(Me[0, 0, 0] - 1.0 / 12.0) < 1e-15
    # curl w_01 = 2 grad lam0 x grad lam1 = 2 (-1,-1,-1) x (1,0,0) = (0,-2,2); |.|^2 = 8
    assert abs(Ke[0, 0, 0] - 8.0 / 6.0) < 1e-14


@pytest.mark.parametrize("n", [2, 3])
def test_constant_and_rotation_fields(n):
    """Constants and a x x lie in the lowest-order Nedelec space, so their DOF vectors
    reproduce int |c|^2, int |a x x|^2 and int |curl|^2 exactly."""
    m = KuhnMesh(n)
    K, M = fem.assemble_full_KM(m)
    xa = m.coords(m.edges[:, 0])
    xb = m.coords(m.edges[:, 1])
    c = np.array([0.3, -1.2, 0.7])
    xc = (xb - xa) @ c
    assert abs(xc @ M @ xc - c @ c) < 1e-12
    assert abs(xc @ K @ xc) < 1e-11
    a = np.array([0.5, 1.5, -0.8])
    mid = 0.5 * (xa + xb)
    xr = np.einsum("ei,ei->e", np.cross(a, mid), xb - xa)
    assert abs(xr @ K @ xr - 4 * a @ a) < 1e-10
    exact = a @ a - (a @ a / 3 + (a.sum() ** 2 - a @ a) / 4)
    assert abs(xr @ M @ xr - exact) < 1e-12


@pytest.mark.parametrize("n", [3, 4])
def test_gradient_kernel(n):
    """K G phi = 0 and A_xi G phi = -(k^2 + i xi) M G phi for interior nodal phi."""
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    G = fem.discrete_gradient(m)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((n + 1) ** 3) * fem.interior_vertices(m)
    u = G @ phi
    assert np.abs(K @ u).max() < 1e-11 * np.abs(K).max() * np.abs(u).max()
    A = fem.a_xi(K, M, 3.0, 2.0)
    assert np.allclose(A @ u, -(9.0 + 2.0j) * (M @ u), atol=1e-12)


def test_symmetry():
    m = KuhnMesh(3)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, 2.0, 5.0)
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()
    assert (M.diagonal() > 0).all()


def test_gauss_legendre_closed_form():
    t, w = fem.gauss_legendre01(3)
    r = math.sqrt(0.6)
    assert np.allclose(t, [(1 - r) / 2, 0.5, (1 + r) / 2], atol=1e-15)
    assert np.allclose(w, [5 / 18, 4 / 9, 5 / 18], atol=1e-15)


@pytest.mark.parametrize("q,deg", [(2, 1), (3, 3), (4, 5)])
def test_duffy_rule_monomials(q, deg):
    """int_T x^a y^b z^c = a! b! c! / (a + b + c + 3)! on the reference tet."""
    xi, w = fem.duffy_rule(q)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                assert abs(got - exact) < 1e-15


@pytest.mark.parametrize("n", [2, 3])
def test_load_vector_constant_field(n):
    """For constant F = c, f_i = int c . w_i = (M_full x_c)_i on interior rows."""
    m = KuhnMesh(n)
    c = np.array([0.2 + 0.1j, -0.4, 1.0j])
    f = fem.load_vector(m, lambda x: np.broadcast_to(c, x.shape).astype(complex))
    K, M = fem.assemble_full_KM(m)
    xa = m.coords(m.edges[:, 0])
    xb = m.coords(m.edges[:, 1])
    g = M @ ((xb - xa) @ c)
    row = {tuple(e): i for i, e in enumerate(m.edges.tolist())}
    rows = [row[tuple(e)] for e in m.dof_edges.tolist()]
    assert np.allclose(f, g[rows], atol=1e-14)


def _manufactured_error(n, k, xi):
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, k, xi)
    pi = math.pi

    def E(x):
        sx, sy, sz = np.sin(pi * x[:, 0]), np.sin(pi * x[:, 1]), np.sin(pi * x[:, 2])
        return np.stack([sy * sz, sx * sz, sx * sy], axis=1).astype(complex)

    s = 2 * pi * pi - k * k - 1j * xi
    f = fem.load_vector(m, lambda x: s * E(x), q=4)
    u = spla.spsolve(A.tocsc(), f)
    # L2 error of E_h = sum u_e w_e with a q=4 rule per tet
    P = m.coords(m.tets)
    G, vol = fem.bary_gradients(P)
    xi_q, wq = fem.duffy_rule(4)
    err2 = 0.0
    for qp in range(xi_q.shape[0]):
        lam = np.concatenate([[1 - xi_q[qp].sum()], xi_q[qp]])
        x = P[:, 0] + np.einsum("m,tmi->ti", xi_q[qp], P[:, 1:] - P[:, :1])
        Eh = np.zeros((P.shape[0], 3), dtype=complex)
        for a, (p, q) in enumerate(LOCAL_EDGES):
            d = m.tet2dof[:, a]
            coef = np.where(d >= 0, u[np.maximum(d, 0)], 0)
            Eh += coef[:, None] * (lam[p] * G[:, q] - lam[q] * G[:, p])
        err2 += np.sum(6 * vol * wq[qp] * np.sum(np.abs(Eh - E(x)) ** 2, axis=1))
    return math.sqrt(err2)


def test_manufactured_first_order():
    e4 = _manufactured_error(4, 2.0, 3.0)
    e8 = _manufactured_error(8, 2.0, 3.0)
    e12 = _manufactured_error(12, 2.0, 3.0)
    r1, r2 = math.log2(e4 / e8), math.log(e8 / e12) / math.log(1.5)
    assert 0.85 < r1 < 1.3 and 0.9 < r2 < 1.2, (e4, e8, e12)


PI = math.pi
_GL_X, _GL_W = np.polynomial.legendre.leggauss(5)


def _E_div_free(x):
    """(sin pi y sin pi z, sin pi x sin pi z, sin pi x sin pi y): zero tangential trace on the
    cube, divergence free, curl curl E = 2 pi^2 E."""
    sx, sy, sz = np.sin(PI * x[:, 0]), np.sin(PI * x[:, 1]), np.sin(PI * x[:, 2])
    return np.stack([sy * sz, sx * sz, sx * sy], axis=1).astype(complex)


def _E_grad(x):
    """grad(sin pi x sin pi y sin pi z): curl free, zero tangential trace (the potential
    vanishes on the boundary)."""
    sx, sy, sz = np.sin(PI * x[:, 0]), np.sin(PI * x[:, 1]), np.sin(PI * x[:, 2])
    cx, cy, cz = np.cos(PI * x[:, 0]), np.cos(PI * x[:, 1]), np.cos(PI * x[:, 2])
    return (PI * np.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz], axis=1)).astype(complex)


def _edge_interpolant(m, E):
    """Degrees of freedom of the edge interpolant: the line integral of E along each DOF edge,
    oriented from the lower to the higher vertex (5-point Gauss-Legendre on the edge)."""
    a, b = m.coords(m.dof_edges[:, 0]), m.coords(m.dof_edges[:, 1])
    t = b - a
    out = np.zeros(len(a), dtype=complex)
    for xq, wq in zip(_GL_X, _GL_W):
        out += 0.5 * wq * np.sum(E(a + 0.5 * (xq + 1.0) * t) * t, axis=1)
    return out


def _solve_manufactured(n, k, xi, E, s):
    """Galerkin solution u of curl curl E - (k^2 + i xi) E = s E (F = s E) on the n^3 mesh,
    with its L2 and curl errors against E (curl E = 0 for the gradient field; for the
    divergence-free field curl is not needed: only the L2 part and the interpolant are used)."""
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, k, xi)
    f = fem.load_vector(m, lambda x: s * E(x), q=4)
    u = spla.spsolve(A.tocsc(), f)
    P = m.coords(m.tets)
    G, vol = fem.bary_gradients(P)
    xq, wq = fem.duffy_rule(4)
    l2, curl2 = 0.0, 0.0
    for qp in range(xq.shape[0]):
        lam = np.concatenate([[1 - xq[qp].sum()], xq[qp]])
        x = P[:, 0] + np.einsum("m,tmi->ti", xq[qp], P[:, 1:] - P[:, :1])
        Eh = np.zeros((P.shape[0], 3), dtype=complex)
        Ch = np.zeros((P.shape[0], 3), dtype=complex)
        for a, (p, q) in enumerate(LOCAL_EDGES):
            d = m.tet2dof[:, a]
            coef = np.where(d >= 0, u[np.maximum(d, 0)], 0)
            Eh += coef[:, None] * (lam[p] * G[:, q] - lam[q] * G[:, p])
            Ch += coef[:, None] * 2.0 * np.cross(G[:, p], G[:, q])
        l2 += np.sum(6 * vol * wq[qp] * np.sum(np.abs(Eh - E(x)) ** 2, axis=1))
        curl2 += np.sum(6 * vol * wq[qp] * np.sum(np.abs(Ch) ** 2, axis=1))
    return m, K, M, u, math.sqrt(l2), math.sqrt(curl2)


def _rates(e, ns):
    return [math.log(e[i] / e[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(len(e) - 1)]


def test_manufactured_gradient_field():
    """E = grad phi, F = -(k^2 + i xi) E: the second manufactured solution. The L2 error and
    the H(curl) error (curl E = 0, so the curl part is ||curl E_h||) converge at first order,
    and ||curl E_h|| itself falls faster than the L2 error."""
    k, xi = 2.0, 3.0
    ns = (4, 8, 12)
    res = [_solve_manufactured(n, k, xi, _E_grad, -(k * k + 1j * xi)) for n in ns]
    l2 = [r[4] for r in res]
    curl = [r[5] for r in res]
    hcurl = [math.hypot(a, b) for a, b in zip(l2, curl)]
    for r in _rates(l2, ns) + _rates(hcurl, ns):
        assert 0.85 < r < 1.3, (l2, curl)
    assert all(r > 1.5 for r in _rates(curl, ns)), curl
    assert all(c < a for c, a in zip(curl, l2))


@pytest.mark.parametrize("field", ["div_free", "grad"])
def test_discrete_solution_is_close_to_the_edge_interpolant(field):
    """Supercloseness on the uniform Kuhn mesh: E_h - Pi_h E (Pi_h the edge interpolant) is
    one order smaller in L2 than E_h - E, i.e. second order, and the largest error in the
    tangential edge averages u_e / |e| - (Pi_h E)_e / |e| tends to second order too. A dropped or mis-scaled term in K, M or the load vector
    leaves an O(1) or first-order discrepancy here."""
    k, xi = 2.0, 3.0
    if field == "div_free":
        E, s = _E_div_free, 2 * PI * PI - k * k - 1j * xi
    else:
        E, s = _E_grad, -(k * k + 1j * xi)
    ns = (4, 8, 12)
    l2, mid = [], []
    for n in ns:
        m, K, M, u, _, _ = _solve_manufactured(n, k, xi, E, s)
        d = u - _edge_interpolant(m, E)
        l2.append(math.sqrt(abs(np.vdot(d, M @ d))))
        L = np.linalg.norm(m.coords(m.dof_edges[:, 1]) - m.coords(m.dof_edges[:, 0]), axis=1)
        mid.append(float(np.max(np.abs(d) / L)))
    for r in _rates(l2, ns):
        assert 1.75 < r < 2.3, (field, l2, mid)
    # the largest edge error is pre-asymptotic on the coarsest mesh (gradient field: 1.63
    # from n = 4 to 8, 1.83 from 8 to 12): above first order at once, near 2 on the finer pair
    rm = _rates(mid, ns)
    assert all(1.55 < r < 2.3 for r in rm) and rm[-1] > 1.75, (field, l2, mid)


def test_load_vector_of_a_gaussian_bump_against_its_integral():
    """Bump field F(x) = p exp(-|x - c|^2 / w^2) (the right-hand sides' definition): for a
    constant direction e, the edge interpolant of e has the DOFs g_i = e . (x_high - x_low) and
    reproduces e exactly, so sum_i f_i g_i = int F . e dx = (p . e) (pi w^2)^(3/2), up to the
    Gaussian's tail outside the cube (exp(-22) here) and the quadrature error."""
    m = KuhnMesh(10)
    c = np.array([[[0.5, 0.47, 0.52]]])
    p = np.array([[[1.0, 2.0j, -0.5]]])
    w = 0.1
    f = fem.load_vector(m, fem.bump_field(c, p, w))[:, 0]
    t = m.coords(m.dof_edges[:, 1]) - m.coords(m.dof_edges[:, 0])
    for e in np.eye(3):
        exact = (p[0, 0] @ e) * (math.pi * w * w) ** 1.5
        assert abs(f @ (t @ e) - exact) <= 5e-6 * abs(exact), e

"""Pins for oracle.dd: local DOF counts (closed form), the cover property, minors equal
the Galerkin matrix of the box with PEC on its boundary (Eq. 3.3 remark), coarse
interpolation commutes with gradients and gives the coarse Galerkin matrix, R^0 = I when
the meshes coincide, idempotent local projections (Lemma 5.1), and B^{-1} = A^{-1} for a
single subdomain."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.mesh import KuhnMesh, count_interior_edges, vertex_ijk
from oracle import fem, dd


@pytest.mark.parametrize("n,core,overlap", [(10, 5, 1), (12, 5, 1), (9, 4, 2), (6, 3, 0)])
def test_local_counts_and_cover(n, core, overlap):
    m = KuhnMesh(n)
    boxes = dd.subdomain_boxes(n, core, overlap)
    assert len(boxes) == (-(-n // core)) ** 3
    cover = np.zeros(m.n_dof, dtype=int)
    for lo, hi in boxes:
        idx = dd.local_dofs(m, lo, hi)
        a, b, c = (hi - lo).tolist()
        assert len(idx) == count_interior_edges(a, b, c)
        assert np.all(np.diff(idx) > 0)
        cover[idx] += 1
    if overlap > 0:
        assert cover.min() >= 1  # I^h = union of I^h(Omega_l) (Sec. 3.1)
    assert cover.max() <= 8


def test_subdomain_sizes_40():
    # 8 x 8 x 8 boxes of 5^3 cells + 1-cell overlap on 40^3 cells: boxes of 6 or 7 cells
    boxes = dd.subdomain_boxes(40, 5, 1)
    sizes = [count_interior_edges(*(hi - lo).tolist()) for lo, hi in boxes]
    assert len(boxes) == 512 and max(sizes) == 1981 and min(sizes) == 1206
    assert sum(sizes) == 902664


def _box_matrix(a, h, k, xi):
    """Galerkin matrix of an a^3 Kuhn box of cell size h with PEC on its boundary."""
    mb = KuhnMesh(a)
    K, M = fem.assemble_KM(mb)
    s = mb.h / h  # K scales like 1/h, M like h
    return fem.a_xi(K * s, M / s, k, xi)


@pytest.mark.parametrize("l", [0, 13, 26])
def test_minor_is_box_galerkin_matrix(l):
    """A^l = R^l A (R^l)^T is the Galerkin matrix of the problem on Omega_l with PEC
    on its boundary (Eq. 3.3 and the remark after it)."""
    n, k, xi = 15, 3.0, 2.0
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, k, xi)
    S = dd.Schwarz(m, A, 5, 1)
    lo, hi = S.boxes[l]
    a = (hi - lo)
    if not np.all(a == a[0]):
        pytest.skip("non-cubic box")
    Ab = _box_matrix(int(a[0]), m.h, k, xi)
    Al = S.minor(l)
    assert abs(Al - Ab).max() < 1e-12 * abs(Ab).max()


def _nodal_prolongation(fine, coarse, phi_c):
    """Values at fine vertices of the coarse P1 function phi_c (barycentric interpolation
    in the coarse Kuhn simplex holding each fine vertex)."""
    m = coarse.n
    H = 1.0 / m
    x = fine.coords(np.arange((fine.n + 1) ** 3))
    s = x / H
    cube = np.clip(np.floor(s + 1e-12).astype(int), 0, m - 1)
    loc = s - cube
    out = np.empty(x.shape[0])
    for i in range(x.shape[0]):
        perm = np.argsort(-loc[i], kind="stable")
        lam = [1 - loc[i][perm[0]], loc[i][perm[0]] - loc[i][perm[1]],
               loc[i][perm[1]] - loc[i][perm[2]], loc[i][perm[2]]]
        v = cube[i].copy()
        vals = [phi_c[v[0] + (m + 1) * (v[1] + (m + 1) * v[2])]]
        for ax in perm:
            v[ax] += 1
            vals.append(phi_c[v[0] + (m + 1) * (v[1] + (m + 1) * v[2])])
        out[i] = np.dot(lam, vals)
    return out


@pytest.mark.parametrize("n,m", [(4, 2), (6, 2), (6, 3)])
def test_coarse_commutes_with_gradient(n, m):
    """(R^0)^T G_c phi = G_f P phi: the coarse gradient interpolates exactly."""
    fine, coarse = KuhnMesh(n), KuhnMesh(m)
    R0 = dd.coarse_restriction(fine, coarse)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((m + 1) ** 3) * fem.interior_vertices(coarse)
    lhs = R0.T @ (fem.discrete_gradient(coarse) @ phi)
    rhs = fem.discrete_gradient(fine) @ _nodal_prolongation(fine, coarse, phi)
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (8, 2)])
def test_coarse_galerkin(n, m):
    """R^0 A_h (R^0)^T equals the matrix assembled on the coarse mesh (nested spaces)."""
    fine, coarse = KuhnMesh(n), KuhnMesh(m)
    R0 = dd.coarse_restriction(fine, coarse)
    Kf, Mf = fem.assemble_KM(fine)
    Kc, Mc = fem.assemble_KM(coarse)
    Af, Ac = fem.a_xi(Kf, Mf, 2.0, 1.0), fem.a_xi(Kc, Mc, 2.0, 1.0)
    G = R0 @ Af @ R0.T
    assert abs(G - Ac).max() < 1e-12 * abs(Ac).max()


def test_coarse_identity():
    m = KuhnMesh(3)
    R0 = dd.coarse_restriction(m, KuhnMesh(3))
    assert abs(R0 - sp.identity(m.n_dof)).max() < 1e-14


def test_local_projection_idempotent():
    """P_l = (R^l)^T (A^l)^{-1} R^l A is a projection when xi_prob = xi_prec (Lemma 5.1)."""
    n = 10
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, 4.0, 4.0)
    S = dd.Schwarz(m, A, 5, 1)
    S.factor()
    rng = np.random.default_rng(2)
    v = rng.standard_normal(m.n_dof) + 1j * rng.standard_normal(m.n_dof)
    for l in (0, 5):
        i = S.idx[l]

        def P(u):
            z = np.zeros_like(u)
            z[i] = S.local_solve(l, (A @ u)[i])
            return z
        p1 = P(v)
        assert np.abs(P(p1) - p1).max() < 1e-10 * np.abs(p1).max()


def test_single_subdomain_is_exact_inverse():
    m = KuhnMesh(4)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, 3.0, 3.0)
    S = dd.Schwarz(m, A, 4, 0)
    assert len(S.idx) == 1 and len(S.idx[0]) == m.n_dof
    S.factor()
    x = np.arange(m.n_dof) * (1 + 0.5j)
    assert np.abs(S.apply(A @ x) - x).max() < 1e-10 * np.abs(x).max()


def test_as_complex_symmetric():
    """B^{-1} is complex symmetric (sum of R^T (A^l)^{-1} R with symmetric A^l)."""
    m = KuhnMesh(10)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, 5.0, 5.0)
    S = dd.Schwarz(m, A, 5, 1, coarse_m=5, k=5.0, xi_prec=5.0)
    S.factor()
    rng = np.random.default_rng(3)
    u = rng.standard_normal(m.n_dof) + 1j * rng.standard_normal(m.n_dof)
    v = rng.standard_normal(m.n_dof) + 1j * rng.standard_normal(m.n_dof)
    a, b = u @ S.apply(v), v @ S.apply(u)
    assert abs(a - b) < 1e-10 * abs(a)


# ---- restricted and hybrid variants (Sec. 6.3) ---------------------------------------
def _rs(n=6, core=3, overlap=1, cm=3):
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, 3.0, 9.0)
    S = dd.Schwarz(m, A, core, overlap, cm, 3.0, 9.0)
    S.factor()
    return m, A, S


def test_partition_of_unity_sums_to_identity():
    """sum_l (R^l)^T D^l R^l = I (the identity that defines D^l in Sec. 6.3): every DOF is
    owned by exactly one subdomain, and that subdomain holds it."""
    for n, core in ((6, 3), (7, 3), (10, 5)):
        m = KuhnMesh(n)
        K, M = fem.assemble_KM(m)
        S = dd.Schwarz(m, fem.a_xi(K, M, 1.0, 1.0), core, 1)
        pou = S.partition_of_unity()
        total = np.zeros(m.n_dof)
        for l, i in enumerate(S.idx):
            total[i[pou[l]]] += 1
        assert np.array_equal(total, np.ones(m.n_dof))


@pytest.mark.parametrize("n,core", [(6, 3), (7, 3), (10, 5), (11, 4)])
def test_each_dof_is_owned_by_the_core_box_holding_its_midpoint(n, core):
    """The reading behind D^l (Sec. 6.3): the owner of a DOF is the subdomain whose core box
    [core i, core (i + 1)) per axis (the last box closed at n) contains the edge midpoint.
    Checked as an inequality on the midpoint's coordinates, with a ragged last box for n = 7, 11."""
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    S = dd.Schwarz(m, fem.a_xi(K, M, 1.0, 1.0), core, 1)
    N = -(-n // core)
    own = S.owner()
    mid = 0.5 * (m.coords(m.dof_edges[:, 0]) + m.coords(m.dof_edges[:, 1]))  # unit-cube coordinates
    box = np.stack([own % N, (own // N) % N, own // (N * N)], axis=1)
    lo = box * core / n
    hi = np.minimum((box + 1) * core, n) / n
    last = box == N - 1
    eps = 1e-12
    assert np.all(mid >= lo - eps)
    assert np.all((mid < hi - eps) | (last & (mid <= hi + eps)))


def test_preconditioner_is_built_from_xi_prec():
    """Sec. 6.2: B^{-1} comes from A_{xi_prec}, the operator is A_{xi_prob}. With one subdomain
    covering the cube B^{-1} = A_{xi_prec}^{-1} exactly, also when xi_prob differs."""
    from oracle.problem import Problem
    for bc in ("pec", "imp"):
        P = Problem(4, 3.0, 0.5, 6.0, 4, 0, bc=bc)
        P.factor()
        A_prec = fem.a_xi(P.K, P.M, 3.0, 6.0, P.B)
        x = np.arange(P.n_dof) * (1 - 0.25j) + 1.0
        assert np.abs(P.dd.apply(A_prec @ x) - x).max() < 1e-10 * np.abs(x).max(), bc
        assert np.abs(P.dd.apply(P.A @ x) - x).max() > 1e-3 * np.abs(x).max(), bc


def test_ras_single_subdomain_is_the_inverse():
    """One subdomain covering the cube: D = I and RAS = AS = A^{-1}."""
    m = KuhnMesh(4)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, 2.0, 4.0)
    S = dd.Schwarz(m, A, 4, 1)
    S.factor()
    v = np.random.default_rng(0).standard_normal(m.n_dof) + 0j
    z = S.apply(v, levels=(1,), kind="ras")
    assert np.allclose(A @ z, v, atol=1e-11 * np.abs(v).max())


def test_ras_restricts_each_local_solution_to_its_owned_dofs():
    """RAS1 v equals the sum of the local solutions masked by D^l, written out DOF by DOF."""
    m, A, S = _rs()
    v = np.random.default_rng(1).standard_normal(m.n_dof) + 1j * np.random.default_rng(2).standard_normal(m.n_dof)
    z = S.apply(v, levels=(1,), kind="ras")
    own = S.owner()
    ref = np.zeros(m.n_dof, dtype=complex)
    for l, i in enumerate(S.idx):
        zl = spla.spsolve(A[i][:, i].tocsc(), v[i])
        for a, dof in enumerate(i):
            if own[dof] == l:
                ref[dof] = zl[a]
    assert np.allclose(z, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_coarse_projection_and_hybrid_identities():
    """With the Galerkin coarse matrix G A is a projection (G A G = G), and both hybrid
    forms reproduce the coarse correction on its range: B^{-1} A G w = G w for Eq. HRAS and
    Eq. ADEF1ras."""
    m, A, S = _rs()
    rng = np.random.default_rng(3)
    w = rng.standard_normal(m.n_dof) + 1j * rng.standard_normal(m.n_dof)
    gw = S.coarse_correction(w)
    scale = np.abs(gw).max()
    assert np.allclose(S.coarse_correction(A @ gw), gw, atol=1e-10 * scale)
    for kind in ("hras", "adef1"):
        z = S.apply(A @ gw, kind=kind)
        assert np.allclose(z, gw, atol=1e-9 * scale), kind


def test_hybrid_forms_against_their_definitions():
    """HRAS and ADEF1 recomposed from dense matrices of G, A and RAS1 (small mesh)."""
    m, A, S = _rs(n=4, core=2, overlap=1, cm=2)
    nd = m.n_dof
    I = np.eye(nd)
    R1 = np.column_stack([S.ras1(I[:, j].astype(complex)) for j in range(nd)])
    G = np.column_stack([S.coarse_correction(I[:, j].astype(complex)) for j in range(nd)])
    Ad = A.toarray()
    v = np.random.default_rng(4).standard_normal(nd) + 0j
    h = (I - G @ Ad) @ R1 @ (I - Ad @ G) + G
    a = R1 @ (I - Ad @ G) + G
    assert np.allclose(S.apply(v, kind="hras"), h @ v, atol=1e-10 * np.abs(h @ v).max())
    assert np.allclose(S.apply(v, kind="adef1"), a @ v, atol=1e-10 * np.abs(a @ v).max())

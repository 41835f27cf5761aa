"""GPU parity for the impedance boundary condition (Eq. imp) and the ImpRAS local problems
(Sec. 6.3) through the C ABI against the oracle: integer mesh and closed-box subdomain data
bit-exact, K, M and the boundary mass B (fine and coarse) and R^0 to rounding, the box
Galerkin matrices and their factors, the operator, every preconditioner variant, and GMRES
with xi_prob = 0 (the paper's impedance experiments), including the inexact coarse solve by
inner GMRES with one-level ImpRAS (Sec. 6.4)."""
import numpy as np
import pytest

import inputs
from oracle.mesh import KuhnMesh
from oracle import fem, dd
from oracle.problem import Problem as OracleProblem
from parity import assert_close, MIXED_APPLY_TOL, TF32_SOLVE_TOL

pytestmark = pytest.mark.gpu

mx = pytest.importorskip("paper_1711_03789_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

IMP = mx.MX_BC_IMPEDANCE


def _h(n, k, xp, xq, core, ov, cm=0, prec=mx.MX_PLAIN_FP64):
    return mx.Problem(n, k, xp, xq, core, ov, cm, prec, bc=IMP)


@pytest.mark.parametrize("n", [1, 2, 5])
def test_mesh_all_edges_bit_exact(n):
    with _h(n, 2.0, 0.0, 0.0, n, 0) as P:
        key, t2d = mx.mx_get_mesh(P.h, n)
    m = KuhnMesh(n, "imp")
    assert np.array_equal(key, m.dof_key.astype(np.int32))
    assert np.array_equal(t2d, m.tet2dof.astype(np.int32))
    assert (t2d >= 0).all()


@pytest.mark.parametrize("n,core,ov", [(10, 5, 1), (9, 4, 2), (6, 3, 0)])
def test_closed_box_lists_bit_exact(n, core, ov):
    with _h(n, 2.0, 0.0, 1.0, core, ov) as P:
        off, lists, iptr, ipos = mx.mx_get_subdomains(P.h)
    m = KuhnMesh(n, "imp")
    exp = [dd.local_dofs(m, lo, hi, closed=True) for lo, hi in dd.subdomain_boxes(n, core, ov)]
    for l, e in enumerate(exp):
        assert np.array_equal(lists[off[l]:off[l + 1]], e.astype(np.int32)), l
    want = [[] for _ in range(m.n_dof)]
    for l, e in enumerate(exp):
        for j, g in enumerate(e):
            want[g].append(off[l] + j)
    assert np.array_equal(np.diff(iptr), [len(w) for w in want])
    assert np.array_equal(ipos, np.concatenate([np.array(w, dtype=np.int32) for w in want]))


@pytest.mark.parametrize("n,cm", [(4, 2), (6, 3)])
def test_assembly_boundary_mass_and_coarse(n, cm):
    with _h(n, 2.0, 0.0, 1.0, n, 0, cm=cm) as P:
        rowptr, col, K, M = mx.mx_get_csr(P.h)
        B = mx.mx_get_boundary_mass(P.h)
        rpc, colc, Kc, Mc = mx.mx_get_csr(P.h, 1)
        Bc = mx.mx_get_boundary_mass(P.h, 1)
        rp0, col0, val0 = mx.mx_get_coarse_restriction(P.h)
    m, mc = KuhnMesh(n, "imp"), KuhnMesh(cm, "imp")
    Ko, Mo = fem.assemble_KM(m)
    Bo = fem.assemble_B(m)
    assert np.array_equal(rowptr, Ko.indptr) and np.array_equal(col, Ko.indices)
    assert np.abs(K - Ko.data).max() <= 1e-14 * np.abs(Ko.data).max()
    assert np.abs(M - Mo.data).max() <= 1e-14 * np.abs(Mo.data).max()
    Bd = Bo.toarray()[np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr)), col]
    assert np.abs(B - Bd).max() <= 1e-14
    assert abs(Bo.sum() - B.sum()) <= 1e-12  # no entry of B outside the K pattern
    Kco, Mco = fem.assemble_KM(mc)
    Bco = fem.assemble_B(mc).toarray()[np.repeat(np.arange(len(rpc) - 1), np.diff(rpc)), colc]
    assert np.array_equal(colc, Kco.indices)
    assert np.abs(Kc - Kco.data).max() <= 1e-14 * np.abs(Kco.data).max()
    assert np.abs(Bc - Bco).max() <= 1e-14
    R0 = dd.coarse_restriction(m, mc)
    R0.data[np.abs(R0.data) < 1e-13] = 0.0
    R0.eliminate_zeros()
    assert np.array_equal(rp0, R0.indptr) and np.array_equal(col0, R0.indices)
    assert np.abs(val0 - R0.data).max() <= 1e-14


@pytest.mark.parametrize("prec", [mx.MX_PLAIN_FP64, mx.MX_MIXED])
@pytest.mark.parametrize("xi", [2.0, 0.0, -1.5])
def test_box_matrices_and_factors(prec, xi):
    """ImpRAS local matrices (box Galerkin, impedance on the whole box surface) and their
    no-pivot LU, against the oracle's box_matrix."""
    n, k = 10, 4.0
    m = KuhnMesh(n, "imp")
    Ko, Mo = fem.assemble_KM(m)
    S = dd.Schwarz(m, fem.a_xi(Ko, Mo, k, xi, fem.assemble_B(m)), 5, 1, k=k, xi_prec=xi)
    with _h(n, k, 0.0, xi, 5, 1, prec=prec) as P:
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 0)
        nl = [len(i) for i in S.idx]
        mats = {l: mx.mx_get_local(P.h, l, nl[l]) for l in (0, 3, 7)}
        P.factor()
        facs = {l: mx.mx_get_local(P.h, l, nl[l]) for l in (0, 3, 7)}
    tol_a = 4e-15 if prec == mx.MX_PLAIN_FP64 else 1e-7
    tol_lu = 1e-12 if prec == mx.MX_PLAIN_FP64 else 2e-5
    for l in mats:
        Al = S.box_matrix(l).toarray()
        scale = np.abs(Al).max()
        assert np.abs(mats[l] - Al).max() <= tol_a * scale, l
        F = facs[l]
        L = np.tril(F, -1) + np.eye(F.shape[0])
        assert np.abs(L @ np.triu(F) - Al).max() <= tol_lu * scale, l


@pytest.mark.parametrize("xi", [0.0, 3.0])
def test_operator(xi):
    n, k = 6, 3.0
    O = OracleProblem(n, k, xi, 1.0, 3, 1, bc="imp")
    x = inputs.random_complex(61, (2, O.n_dof))
    with _h(n, k, xi, 1.0, 3, 1) as P:
        y = mx.mx_spmv(P.h, x)
    ye = (O.A @ x.T).T
    assert np.abs(y - ye).max() <= 1e-13 * np.abs(ye).max()


@pytest.mark.parametrize("prec", [mx.MX_PLAIN_FP64, mx.MX_MIXED])
@pytest.mark.parametrize("kind,name", [(mx.MX_PREC_AS, "as"), (mx.MX_PREC_RAS, "ras"), (mx.MX_PREC_HRAS, "hras"),
                                       (mx.MX_PREC_ADEF1, "adef1")])
def test_preconditioners(prec, kind, name):
    """ImpAS, ImpRAS, ImpHRAS and ADEF1-ImpRAS applies (two-level, impedance coarse
    problem) against the oracle."""
    n, k, xi = 10, 5.0, 5.0
    O = OracleProblem(n, k, 0.0, xi, 5, 1, coarse_m=5, kind=name, bc="imp")
    O.factor()
    v = inputs.random_complex(67, (3, O.n_dof))
    with _h(n, k, 0.0, xi, 5, 1, cm=5, prec=prec) as P:
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 0)
        P.factor()
        mx.mx_set_preconditioner(P.h, kind)
        z = P.precond(v, levels=3)
    ze = O.dd.apply(v.T, levels=(1, 0), kind=name).T
    tol = 1e-11 if prec == mx.MX_PLAIN_FP64 else MIXED_APPLY_TOL
    assert_close(z, ze, tol, what=f"impedance {name} apply")


@pytest.mark.parametrize("prec", [mx.MX_PLAIN_FP64, mx.MX_MIXED])
@pytest.mark.parametrize("xi_prec", [0.0, 6.0])
def test_gmres_impedance_hras(prec, xi_prec):
    """xi_prob = 0 with the impedance condition and ImpHRAS (the paper's Table 7 setting;
    xi_prec = 0 there, k in its preliminary runs): the oracle's solution to 1e-8 and, in the
    FP64 form, the same iteration count (+-1)."""
    n, k, nrhs = 10, 6.0, 2
    c, p = inputs.bump_batch(11, nrhs)
    O = OracleProblem(n, k, 0.0, xi_prec, 5, 1, coarse_m=5, kind="hras", bc="imp")
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-10, max_it=300)
    with _h(n, k, 0.0, xi_prec, 5, 1, cm=5, prec=prec) as P:
        P.factor()
        mx.mx_set_preconditioner(P.h, mx.MX_PREC_HRAS)
        f = P.load_vector(c, p, 0.1)
        assert np.abs(f.T - fo).max() <= 1e-12 * np.abs(fo).max()
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK
    assert_close(x, xo.T, 1e-8, what="impedance GMRES solution")
    for r in range(nrhs):
        assert st[r]["converged"]
        res = np.linalg.norm(fo[:, r] - O.A @ x[r]) / np.linalg.norm(fo[:, r])
        assert res <= 1.05e-10
        if prec == mx.MX_PLAIN_FP64:
            assert abs(st[r]["iterations"] - ost[r][0]) <= 1, (st[r], ost[r])


def test_adef1_impras_with_inner_impras_coarse_solve():
    """The COBRA combination of Sec. 6.4: xi_prob = 0, xi_prec = k, ADEF1-ImpRAS outside,
    the coarse problem by inner GMRES (1e-1) with one-level ImpRAS."""
    n, k, cm = 12, 6.0, 6
    c, p = inputs.bump_batch(13, 1)
    inner = dict(core=2, overlap=1, tol=0.1, max_it=100, kind="ras")
    O = OracleProblem(n, k, 0.0, k, 4, 1, coarse_m=cm, kind="adef1", inner_coarse=inner, bc="imp")
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo[:, 0], tol=1e-10, max_it=300)
    with _h(n, k, 0.0, k, 4, 1, cm=cm) as P:
        P.set_coarse_solver(mx.MX_COARSE_GMRES, core_cells=2, overlap_cells=1, tol=0.1, max_it=100,
                            prec_kind=mx.MX_PREC_RAS)
        P.factor()
        mx.mx_set_preconditioner(P.h, mx.MX_PREC_ADEF1)
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK and st[0]["converged"]
    assert_close(x[0], xo, 1e-8, what="ADEF1-ImpRAS with inner coarse GMRES")
    assert abs(st[0]["iterations"] - ost[0][0]) <= 1


def test_xi_prec_zero_needs_impedance():
    with pytest.raises(mx.MxError) as e:
        mx.Problem(4, 2.0, 0.0, 0.0, 2, 1, 0, mx.MX_PLAIN_FP64)
    assert e.value.code == mx.MX_EINVAL
    with _h(4, 2.0, 0.0, 0.0, 2, 1) as P:
        assert P.n_dof == KuhnMesh(4, "imp").n_dof

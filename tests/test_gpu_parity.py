"""GPU parity: every step of the path through the C ABI against the CPU oracle.

Integer work (mesh, DOF numbering, subdomain lists, inverse map, CSR patterns) must be
bit-exact; FP64 values within a few ulps of the matrix scale; mixed-precision results
within bounds derived from c64 rounding; GMRES solutions within 1e-8 (plain) of the
oracle when both run to a 1e-10 relative residual."""
import numpy as np
import pytest

import inputs
from oracle.mesh import KuhnMesh
from oracle import fem, dd
from oracle.problem import Problem as OracleProblem
from parity import assert_close, MIXED_APPLY_TOL, TF32_SOLVE_TOL, LOAD_DF_TOL

pytestmark = pytest.mark.gpu

mx = pytest.importorskip("paper_1711_03789_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _handle(n, k, xp, xq, core, ov, cm=0, prec=mx.MX_PLAIN_FP64):
    return mx.Problem(n, k, xp, xq, core, ov, cm, prec)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 10])
def test_mesh_integers_bit_exact(n):
    with _handle(n, 2.0, 1.0, 1.0, max(1, n), 0) as P:
        key, t2d = mx.mx_get_mesh(P.h, n)
    m = KuhnMesh(n)
    assert np.array_equal(key, m.dof_key.astype(np.int32))
    assert np.array_equal(t2d, m.tet2dof.astype(np.int32))


@pytest.mark.parametrize("n,core,ov", [(10, 5, 1), (12, 5, 1), (9, 4, 2), (6, 3, 0), (7, 7, 0)])
def test_subdomain_lists_bit_exact(n, core, ov):
    with _handle(n, 2.0, 1.0, 1.0, core, ov) as P:
        off, lists, iptr, ipos = mx.mx_get_subdomains(P.h)
    m = KuhnMesh(n)
    boxes = dd.subdomain_boxes(n, core, ov)
    assert len(off) == len(boxes) + 1
    exp = [dd.local_dofs(m, lo, hi) for lo, hi in boxes]
    for l, e in enumerate(exp):
        assert np.array_equal(lists[off[l]:off[l + 1]], e.astype(np.int32)), l
    # inverse map: positions of each DOF in increasing subdomain order
    want = [[] for _ in range(m.n_dof)]
    for l, e in enumerate(exp):
        for j, g in enumerate(e):
            want[g].append(off[l] + j)
    assert np.array_equal(np.diff(iptr), [len(w) for w in want])
    assert np.array_equal(ipos, np.concatenate([np.array(w, dtype=np.int32) for w in want]))


@pytest.mark.parametrize("n", [2, 6, 10])
def test_assembly(n):
    with _handle(n, 2.0, 1.0, 1.0, n, 0) as P:
        rowptr, col, K, M = mx.mx_get_csr(P.h)
    m = KuhnMesh(n)
    Ko, Mo = fem.assemble_KM(m)
    assert np.array_equal(rowptr, Ko.indptr) and np.array_equal(col, Ko.indices)
    assert np.array_equal(Mo.indptr, Ko.indptr) and np.array_equal(Mo.indices, Ko.indices)
    assert np.abs(K - Ko.data).max() <= 1e-14 * np.abs(Ko.data).max()
    assert np.abs(M - Mo.data).max() <= 1e-14 * np.abs(Mo.data).max()


@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (10, 5), (8, 2)])
def test_coarse_restriction(n, m):
    with _handle(n, 2.0, 1.0, 1.0, n, 0, cm=m) as P:
        rp, col, val = mx.mx_get_coarse_restriction(P.h)
        rpc, colc, Kc, Mc = mx.mx_get_csr(P.h, 1)
    R0 = dd.coarse_restriction(KuhnMesh(n), KuhnMesh(m))
    R0.data[np.abs(R0.data) < 1e-13] = 0.0  # rounding residue where the exact entry is 0
    R0.eliminate_zeros()
    assert np.array_equal(rp, R0.indptr) and np.array_equal(col, R0.indices)
    assert np.abs(val - R0.data).max() <= 1e-14
    Ko, Mo = fem.assemble_KM(KuhnMesh(m))
    assert np.array_equal(colc, Ko.indices)
    assert np.abs(Kc - Ko.data).max() <= 1e-14 * np.abs(Ko.data).max()


@pytest.mark.parametrize("prec,tol", [(mx.MX_PLAIN_FP64, 1e-13), (mx.MX_MIXED, LOAD_DF_TOL)])
@pytest.mark.parametrize("n,nrhs", [(4, 1), (10, 3)])
def test_load_vector(n, nrhs, prec, tol):
    c, p = inputs.bump_batch(11, nrhs)
    with _handle(n, 2.0, 1.0, 1.0, n, 0, prec=prec) as P:
        f = P.load_vector(c, p, 0.1)
        fd = torch.zeros((nrhs, P.n_dof), dtype=torch.complex128, device="cuda")
        P.load_vector(c, p, 0.1, out=fd)
    fo = fem.load_vector(KuhnMesh(n), fem.bump_field(c, p, 0.1))
    err = np.abs(f.T - fo).max() / np.abs(fo).max()
    print(f"load vector n={n} prec={prec}: max error / max|f| = {err:.2e} (bound {tol:.1e})")
    assert err <= tol
    assert np.array_equal(fd.cpu().numpy(), f)


def test_load_vector_in_chunks():
    """40^3 cells, 16 right-hand sides: the tetrahedron contributions of both forms are held
    for 14 right-hand sides at a time (a 512 MB cap), so the batch runs in two chunks. The
    first and last right-hand sides against the oracle, every right-hand side of the mixed form
    against the FP64 form."""
    n, nrhs = 40, 16
    c, p = inputs.bump_batch(11, nrhs)
    f = {}
    for prec in (mx.MX_PLAIN_FP64, mx.MX_MIXED):
        with _handle(n, 2.0, 1.0, 1.0, 8, 0, prec=prec) as P:
            f[prec] = P.load_vector(c, p, 0.1)
    sel = [0, nrhs - 1]
    fo = fem.load_vector(KuhnMesh(n), fem.bump_field(c[sel], p[sel], 0.1))
    scale = np.abs(fo).max()
    assert np.abs(f[mx.MX_PLAIN_FP64][sel].T - fo).max() <= 1e-13 * scale
    assert np.abs(f[mx.MX_MIXED][sel].T - fo).max() <= LOAD_DF_TOL * scale
    d = np.abs(f[mx.MX_MIXED] - f[mx.MX_PLAIN_FP64]).max(axis=1) / np.abs(f[mx.MX_PLAIN_FP64]).max(axis=1)
    print("mixed vs FP64 load vector, per right-hand side:", d.max())
    assert d.max() <= LOAD_DF_TOL


@pytest.mark.parametrize("n,nrhs,xi", [(5, 1, 0.0), (10, 4, 3.0), (12, 16, -2.0)])
def test_spmv(n, nrhs, xi):
    k = 3.0
    x = inputs.random_complex(5, (nrhs, KuhnMesh(n).n_dof))
    with _handle(n, k, xi, 1.0, 5, 1) as P:
        y = P.spmv(x)
        yd = P.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    Ko, Mo = fem.assemble_KM(KuhnMesh(n))
    A = fem.a_xi(Ko, Mo, k, xi)
    ye = (A @ x.T).T
    assert np.abs(y - ye).max() <= 1e-13 * np.abs(ye).max()
    assert np.array_equal(y, yd)


@pytest.mark.parametrize("n,nrhs,xi", [(5, 1, 0.0), (10, 3, 3.0), (10, 2, 1.0), (12, 16, -2.0)])
def test_spmv_mixed(n, nrhs, xi):
    """The double-float operator product of the mixed form (one right-hand side per thread for
    an odd count, pairs for an even one, as in the solver) against the oracle's FP64 operator on
    the same c64-rounded vectors, element by element. Bound per entry: each product carries the
    coefficient's split error (2^-48) and the compensated row sum a few units of 2^-48 of every
    term, so |y - A x|_i <= 2^-44 (|A| |x|)_i; the two FP64 assemblies differ by rounding only."""
    k = 3.0
    x = inputs.random_complex(17, (nrhs, KuhnMesh(n).n_dof))
    x64 = x.astype(np.complex64).astype(np.complex128)
    with _handle(n, k, xi, 1.0, 5, 1, prec=mx.MX_MIXED) as P:
        y = P.spmv_mixed(x)
        yd = P.spmv_mixed(torch.from_numpy(x).cuda()).cpu().numpy()
    Ko, Mo = fem.assemble_KM(KuhnMesh(n))
    A = fem.a_xi(Ko, Mo, k, xi).tocsr()
    ye = (A @ x64.T).T
    bound = 2.0 ** -44 * (abs(A) @ np.abs(x64).T).T
    worst = (np.abs(y - ye) / bound).max()
    print(f"mixed SpMV n={n} nrhs={nrhs}: max |error| / bound = {worst:.3f}")
    assert worst <= 1.0
    assert np.array_equal(y, yd)


@pytest.mark.parametrize("prec", [mx.MX_PLAIN_FP64, mx.MX_MIXED])
def test_local_minor_and_factor(prec):
    n, k, xi = 10, 4.0, 4.0
    m = KuhnMesh(n)
    Ko, Mo = fem.assemble_KM(m)
    A = fem.a_xi(Ko, Mo, k, xi)
    S = dd.Schwarz(m, A, 5, 1)
    with _handle(n, k, 0.0, xi, 5, 1, prec=prec) as P:
        nl = [len(i) for i in S.idx]
        minors = {l: mx.mx_get_local(P.h, l, nl[l]) for l in (0, 3, 7)}
        P.factor()
        factors = {l: mx.mx_get_local(P.h, l, nl[l]) for l in (0, 3, 7)}
    tol_a = 4e-15 if prec == mx.MX_PLAIN_FP64 else 1e-7
    tol_lu = 1e-12 if prec == mx.MX_PLAIN_FP64 else 2e-5
    for l in minors:
        Al = S.minor(l).toarray()
        scale = np.abs(Al).max()
        assert np.abs(minors[l] - Al).max() <= tol_a * scale
        F = factors[l]
        L = np.tril(F, -1) + np.eye(F.shape[0])
        U = np.triu(F)
        assert np.abs(L @ U - Al).max() <= tol_lu * scale


@pytest.mark.parametrize("prec,levels,nrhs", [(mx.MX_PLAIN_FP64, 1, 1), (mx.MX_PLAIN_FP64, 3, 3),
                                              (mx.MX_MIXED, 1, 2), (mx.MX_MIXED, 3, 16),
                                              (mx.MX_PLAIN_FP64, 2, 2)])
def test_preconditioner_apply(prec, levels, nrhs):
    n, k, xi = 10, 5.0, 5.0
    O = OracleProblem(n, k, 0.0, xi, 5, 1, coarse_m=5)
    O.factor()
    v = inputs.random_complex(9, (nrhs, O.n_dof))
    lv = tuple(x for x, bit in ((1, 1), (0, 2)) if levels & bit)
    ze = O.dd.apply(v.T, levels=lv).T
    with _handle(n, k, 0.0, xi, 5, 1, cm=5, prec=prec) as P:
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 0)  # FP32 CUDA-core local solves
        P.factor()
        z = P.precond(v, levels=levels)
    tol = 1e-11 if prec == mx.MX_PLAIN_FP64 else MIXED_APPLY_TOL
    assert_close(z, ze, tol, what=f"apply levels={levels}")


@pytest.mark.parametrize("prec,cm,nrhs", [(mx.MX_PLAIN_FP64, 0, 1), (mx.MX_PLAIN_FP64, 5, 2),
                                          (mx.MX_MIXED, 0, 1), (mx.MX_MIXED, 5, 3)])
def test_gmres_matches_oracle(prec, cm, nrhs):
    """Config-1 problem (10^3 cells, k = xi = 6, 2x2x2 subdomains): both sides to 1e-10."""
    n, k = 10, 6.0
    c, p = inputs.bump_batch(1, nrhs)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=cm)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-10, restart=0, max_it=300)
    with _handle(n, k, k, k, 5, 1, cm=cm, prec=prec) as P:
        P.factor()
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK
    assert_close(x, xo.T, 1e-8, what="GMRES solution")
    for r in range(nrhs):
        assert st[r]["converged"]
        res = np.linalg.norm(fo[:, r] - O.A @ x[r]) / np.linalg.norm(fo[:, r])
        assert res <= 1.05e-10, res
        if prec == mx.MX_PLAIN_FP64:
            assert abs(st[r]["iterations"] - ost[r][0]) <= 1, (st[r], ost[r])


def test_restarted_gmres():
    n, k = 10, 6.0
    c, p = inputs.bump_batch(2, 2)
    O = OracleProblem(n, k, k, k, 5, 1)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-9, restart=20, max_it=400)
    with _handle(n, k, k, k, 5, 1) as P:
        P.factor()
        x, st, rc = P.solve(fo.T.copy(), tol=1e-9, restart=20, max_it=400)
    assert rc == mx.MX_OK
    assert_close(x, xo.T, 1e-7, what="restarted GMRES solution")
    for r in range(2):
        assert abs(st[r]["iterations"] - ost[r][0]) <= 2


def test_single_subdomain_one_iteration():
    """One subdomain covering the cube with xi_prob = xi_prec: B^{-1} = A^{-1}."""
    n, k = 4, 3.0
    with _handle(n, k, k, k, 4, 0) as P:
        P.factor()
        b = inputs.random_complex(3, (1, P.n_dof))
        x, st, rc = P.solve(b, tol=1e-10, max_it=10)
    assert rc == mx.MX_OK and st[0]["iterations"] == 1


def test_zero_rhs_and_errors():
    with _handle(4, 3.0, 3.0, 3.0, 2, 1) as P:
        with pytest.raises(mx.MxError) as e:
            P.solve(np.ones((1, P.n_dof), dtype=np.complex128))
        assert e.value.code == mx.MX_ENOTFACTORED
        P.factor()
        x, st, rc = P.solve(np.zeros((2, P.n_dof), dtype=np.complex128))
        assert rc == mx.MX_OK and np.all(x == 0) and st[0]["iterations"] == 0


def test_nonconvergence_reports_enoconv():
    n, k = 10, 6.0
    with _handle(n, k, 0.0, k, 5, 1) as P:
        P.factor()
        b = inputs.random_complex(4, (1, P.n_dof))
        x, st, rc = P.solve(b, tol=1e-14, max_it=3)
    assert rc == mx.MX_ENOCONV and st[0]["iterations"] == 3 and not st[0]["converged"]
    assert np.isfinite(x).all()


def test_single_dof_mesh():
    with _handle(1, 2.0, 1.0, 1.0, 1, 0) as P:
        assert P.n_dof == 1
        P.factor()
        x, st, rc = P.solve(np.array([[1.0 + 1.0j]]), tol=1e-12)
        A = fem.a_xi(*fem.assemble_KM(KuhnMesh(1)), 2.0, 1.0).toarray()
        assert abs(x[0, 0] - (1 + 1j) / A[0, 0]) < 1e-14


@pytest.mark.parametrize("nvec,n,nrhs", [(1, 7, 1), (5, 40001, 3), (12, 100000, 16)])
def test_batched_dots(nvec, n, nrhs):
    """mx_dots against the definition h[i, r] = sum_x conj(V[i, x, r]) w[x, r] in FP64."""
    V = inputs.random_complex(21, (nvec, n, nrhs))
    w = inputs.random_complex(22, (n, nrhs))
    he = np.einsum("ixr,xr->ir", V.conj(), w)
    h = mx.mx_dots(torch.from_numpy(V).cuda(), torch.from_numpy(w).cuda())
    assert np.abs(h - he).max() <= 1e-13 * np.sqrt(n) * np.abs(V).max() * np.abs(w).max()
    hd = torch.zeros((nvec, nrhs), dtype=torch.complex128, device="cuda")
    mx.mx_dots(torch.from_numpy(V).cuda(), torch.from_numpy(w).cuda(), hd)
    assert np.array_equal(hd.cpu().numpy(), h)


@pytest.mark.parametrize("mode,tol", [(4, 2e-5), (3, 2e-5), (1, 5e-3), (2, 2e-5), (0, 2e-5)])
def test_local_factor_tensor_core_modes(mode, tol):
    """FP32 local LU, one launch per block step with the trailing update on CUDA cores (4),
    tcgen05 3 x TF32 (3) or tcgen05 TF32 (1), and the persistent one-CTA-per-subdomain LU with
    3 x TF32 tcgen05 updates (2, and the default 0): L U reproduces the minor to the
    precision of each mode."""
    n, k, xi = 10, 4.0, 16.0
    m = KuhnMesh(n)
    Ko, Mo = fem.assemble_KM(m)
    A = fem.a_xi(Ko, Mo, k, xi)
    S = dd.Schwarz(m, A, 5, 1)
    with _handle(n, k, 0.0, xi, 5, 1, prec=mx.MX_MIXED) as P:
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LU_TENSOR, mode)
        P.factor()
        for l in (0, 5):
            F = mx.mx_get_local(P.h, l, len(S.idx[l]))
            L = np.tril(F, -1) + np.eye(F.shape[0])
            Al = S.minor(l).toarray()
            assert np.abs(L @ np.triu(F) - Al).max() <= tol * np.abs(Al).max()


def test_fused_local_factor_full_boxes():
    """The persistent tensor-core LU (MX_TUNE_LU_TENSOR = 2, the default) on 20^3 cells: interior boxes of
    7^3 cells (n_l = 1981, half-bandwidth about 350, so three 128-row tiles per window and a
    ragged last tile) and boundary boxes; L U against the oracle's minors (backward error 2e-5,
    as for the per-step LU), and the factors against those of the per-step CUDA-core LU of the
    same c64 minor. The two orders of FP32 arithmetic (panels from inverted diagonal blocks
    against substitution) give factors that differ by rounding carried along the elimination,
    a few times 1e-5 of the largest entry here; bound 2e-4."""
    n, k, xi = 20, 10.0, 100.0
    m = KuhnMesh(n)
    Ko, Mo = fem.assemble_KM(m)
    A = fem.a_xi(Ko, Mo, k, xi)
    S = dd.Schwarz(m, A, 5, 1)
    subs = (0, 21, 63)
    out = {}
    for mode in (2, 4):
        with _handle(n, k, 0.0, xi, 5, 1, prec=mx.MX_MIXED) as P:
            mx.mx_set_tuning(P.h, mx.MX_TUNE_LU_TENSOR, mode)
            P.factor()
            out[mode] = {l: mx.mx_get_local(P.h, l, len(S.idx[l])) for l in subs}
    for l in subs:
        Al = S.minor(l).toarray()
        for mode in (2, 4):
            F = out[mode][l]
            L = np.tril(F, -1) + np.eye(F.shape[0])
            be = np.abs(L @ np.triu(F) - Al).max() / np.abs(Al).max()
            print(f"subdomain {l} mode {mode}: backward error {be:.2e}")
            assert be <= 2e-5, (l, mode, be)
        F, G = out[2][l], out[4][l]
        d = np.abs(F - G).max() / np.abs(G).max()
        print(f"subdomain {l}: factor difference {d:.2e}")
        assert d <= 2e-4, (l, d)


@pytest.mark.parametrize("n,nrhs,after", [(10, 1, False), (10, 16, True), (20, 16, False), (20, 20, False),
                                          (20, 32, True)])
def test_local_solves_tensor_cores(n, nrhs, after):
    """Local solves on tcgen05 (TF32 panels of the c64 factors, right-hand-side block as a
    TF32 hi + lo pair) against the oracle's pivoted dense local solves. At n = 20 the local
    matrices have about 2000 rows, so the 512-slot accumulator ring wraps several times;
    nrhs = 20 leaves a ragged group of 32. `after` switches the mode after factor (panel
    images built at the first solve). Bound: the factors enter rounded to TF32 (unit
    roundoff u = 2^-12 relative), so the solves carry a perturbation of a few u; the test
    allows 4 u per right-hand side, element-wise too (measured: under 2 u)."""
    k, xi = 10.0, 100.0
    O = OracleProblem(n, k, 0.0, xi, 5, 1)
    O.factor()
    v = inputs.random_complex(11, (nrhs, O.n_dof))
    ze = O.dd.apply(v.T, levels=(1,)).T
    with _handle(n, k, 0.0, xi, 5, 1, prec=mx.MX_MIXED) as P:
        if not after:
            mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 1)
        P.factor()
        if after:
            mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 1)
        z = P.precond(v, levels=1)
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 0)
        zc = P.precond(v, levels=1)
    assert_close(z, ze, TF32_SOLVE_TOL, what="tensor-core local solves")
    assert_close(zc, ze, MIXED_APPLY_TOL, what="CUDA-core c64 local solves")


def test_gmres_with_the_fused_tensor_core_factorisation():
    """Mixed-form GMRES on factors from the persistent tensor-core LU reaches the oracle's
    solution (both to 1e-10)."""
    n, k, nrhs = 10, 6.0, 2
    c, p = inputs.bump_batch(4, nrhs)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=5)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-10, restart=0, max_it=300)
    with _handle(n, k, k, k, 5, 1, cm=5, prec=mx.MX_MIXED) as P:
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LU_TENSOR, 2)
        P.factor()
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK and all(v["converged"] for v in st)
    assert_close(x, xo.T, 1e-8, what="GMRES solution, fused tensor-core LU")


def test_gmres_tensor_core_local_solves():
    """FGMRES with the tensor-core local solves reaches the same solution as the oracle.
    The TF32 panels perturb the preconditioner by a few 2^-12 relative, which FGMRES
    absorbs with a few more iterations at a 1e-10 tolerance (bound: 25 % more)."""
    n, k, nrhs = 10, 6.0, 3
    c, p = inputs.bump_batch(1, nrhs)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=5)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-10, restart=0, max_it=300)
    with _handle(n, k, k, k, 5, 1, cm=5, prec=mx.MX_MIXED) as P:
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 1)
        P.factor()
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK
    assert_close(x, xo.T, 1e-8, what="GMRES solution, tensor-core local solves")
    for r in range(nrhs):
        assert st[r]["converged"]
        assert st[r]["iterations"] <= 1.25 * ost[r][0], (st[r], ost[r])


def test_mixed_gmres_16_rhs_matches_oracle():
    """The benchmark's launch configuration on a 20^3 mesh (64 subdomains, a 4^3 coarse mesh,
    k = 10, xi_prob = xi_prec = k^2): 16 right-hand sides in one batched mixed-form solve --
    tensor-core local solves in one 16-wide group, the RHS-paired double-float Gram-Schmidt,
    normalisation and update kernels, the c64 coarse inverse -- against the oracle's FP64
    one-at-a-time solves, both to a 1e-10 relative residual: every solution element by
    element, and iteration counts within 10 % (FGMRES absorbs the c64 / TF32 preconditioner
    with at most a few more iterations)."""
    n, k, nrhs, cm = 20, 10.0, 16, 4
    xi = k * k
    c, p = inputs.bump_batch(1, nrhs)
    O = OracleProblem(n, k, xi, xi, 5, 1, coarse_m=cm)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-10, restart=0, max_it=300)
    with _handle(n, k, xi, xi, 5, 1, cm=cm, prec=mx.MX_MIXED) as P:
        P.factor()
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK
    assert_close(x, xo.T, 1e-8, what="mixed GMRES, 16 right-hand sides")
    for r in range(nrhs):
        assert st[r]["converged"]
        res = np.linalg.norm(fo[:, r] - O.A @ x[r]) / np.linalg.norm(fo[:, r])
        assert res <= 1.05e-10, (r, res)
        assert abs(st[r]["iterations"] - ost[r][0]) <= max(2, 0.1 * ost[r][0]), (r, st[r], ost[r])


@pytest.mark.parametrize("nrhs,n,k,core,cm", [(2, 4, 3.0, 2, 0), (8, 10, 6.0, 5, 5), (16, 12, 8.0, 3, 0),
                                              (32, 12, 8.0, 3, 0)])
def test_staged_second_pass(nrhs, n, k, core, cm):
    """The staged double-float second Gram-Schmidt pass (basis tiles of 8 vectors brought into
    shared-memory stages by bulk copies, one thread per row and right-hand-side pair; the default
    for 2, 4, 8, 16 and 32 right-hand sides) against the lane-parallel kernel: both runs reach a
    1e-12 FP64 true residual on the oracle's operator, so the staged inner products carry the
    full double-float accuracy; their solutions agree element by element, their iteration counts
    within one. Every case runs more than 8 iterations, so the rows are swept once per chunk of 8
    vectors; the cases cover one pair per row (2 right-hand sides, 128 rows per stage), ragged
    last stages, blocks without rows (316 DOFs over two blocks per SM) and the widest batch."""
    c, p = inputs.bump_batch(5, nrhs)
    O = OracleProblem(n, k, k, k, core, 1, coarse_m=cm)
    fo = O.load_vector(c, p, 0.1)
    runs = {}
    for mode in (0, 1):
        with _handle(n, k, k, k, core, 1, cm=cm, prec=mx.MX_MIXED) as P:
            mx.mx_set_tuning(P.h, mx.MX_TUNE_DOTS, mode)
            P.factor()
            f = P.load_vector(c, p, 0.1)
            x, st, rc = P.solve(f, tol=1e-12, restart=0, max_it=400)
        assert rc == mx.MX_OK
        for r in range(nrhs):
            assert st[r]["converged"], (mode, r, st[r])
            res = np.linalg.norm(fo[:, r] - O.A @ x[r]) / np.linalg.norm(fo[:, r])
            assert res <= 1.05e-12, (mode, r, res)
        runs[mode] = (x, np.array([s["iterations"] for s in st]))
    assert runs[0][1].max() > 8, runs[0][1]  # several chunks of vectors
    assert_close(runs[0][0], runs[1][0], 1e-9, what="staged vs lane-parallel second pass")
    assert np.abs(runs[0][1] - runs[1][1]).max() <= 1, (runs[0][1], runs[1][1])


def test_mixed_gmres_tight_tolerance():
    """The mixed form carries its Krylov basis, inner products and operator in double-float
    arithmetic (about 48 bits): it still reaches a 1e-12 FP64 true residual, and its solution
    agrees with the oracle's to the accuracy that residual implies."""
    n, k, nrhs = 10, 6.0, 2
    c, p = inputs.bump_batch(3, nrhs)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=5)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-13, restart=0, max_it=300)
    with _handle(n, k, k, k, 5, 1, cm=5, prec=mx.MX_MIXED) as P:
        P.factor()
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-12, restart=0, max_it=300)
    assert rc == mx.MX_OK
    for r in range(nrhs):
        assert st[r]["converged"] and st[r]["rel_residual"] <= 1e-12
        res = np.linalg.norm(fo[:, r] - O.A @ x[r]) / np.linalg.norm(fo[:, r])
        assert res <= 1.05e-12, res
    assert_close(x, xo.T, 1e-9, what="mixed GMRES at 1e-12")


@pytest.mark.parametrize("n,cm,nrhs", [(10, 5, 3), (20, 10, 16), (20, 4, 20)])
def test_coarse_inverse_apply(n, cm, nrhs):
    """Mixed-form coarse solve with the explicit c64 inverse of A^0 against the oracle's
    pivoted sparse coarse solve (levels = 2: coarse correction only), and against the band
    sweeps of the same c64 factors. The inverse carries the rounding of the c64 factors, and
    the dense product runs on the tensor cores (mode 1: three TF32 products per term; n_c = 6,130
    with one group of 16 right-hand sides, n_c = 316 with a group of 16 and one of 4; n_c = 665
    is odd and takes the CUDA cores) or on the CUDA cores (mode 2, FP32): the bound of the other
    c64 preconditioner parts (MIXED_APPLY_TOL)."""
    k, xi = 6.0, 36.0
    O = OracleProblem(n, k, 0.0, xi, 5, 1, coarse_m=cm)
    O.factor()
    v = inputs.random_complex(21, (nrhs, O.n_dof))
    ze = O.dd.apply(v.T, levels=(0,)).T
    out = {}
    for mode in (1, 2, 0):
        with _handle(n, k, 0.0, xi, 5, 1, cm=cm, prec=mx.MX_MIXED) as P:
            mx.mx_set_tuning(P.h, mx.MX_TUNE_COARSE_INVERSE, mode)
            P.factor()
            out[mode] = P.precond(v, levels=2)
    for mode in (1, 2, 0):
        assert_close(out[mode], ze, MIXED_APPLY_TOL, what=f"coarse apply, inverse={mode}")
    assert_close(out[1], out[0], MIXED_APPLY_TOL, what="inverse against band sweeps")
    assert_close(out[1], out[2], MIXED_APPLY_TOL, what="tensor-core against CUDA-core dense product")


@pytest.mark.parametrize("prec", [mx.MX_PLAIN_FP64, mx.MX_MIXED])
@pytest.mark.parametrize("kind,name", [(mx.MX_PREC_RAS, "ras"), (mx.MX_PREC_HRAS, "hras"),
                                       (mx.MX_PREC_ADEF1, "adef1")])
def test_restricted_and_hybrid_preconditioners(prec, kind, name):
    """RAS (one and two level), HRAS and ADEF1-RAS (Sec. 6.3) against the oracle's
    definitions; bounds as for the additive form (FP64: rounding; mixed: c64 local and
    coarse solves, CUDA-core local solves here)."""
    n, k, xi = 10, 5.0, 25.0
    O = OracleProblem(n, k, 0.0, xi, 5, 1, coarse_m=5)
    O.factor()
    nrhs = 3
    v = inputs.random_complex(31, (nrhs, O.n_dof))
    with _handle(n, k, 0.0, xi, 5, 1, cm=5, prec=prec) as P:
        mx.mx_set_tuning(P.h, mx.MX_TUNE_LOCAL_TENSOR, 0)
        P.factor()
        mx.mx_set_preconditioner(P.h, kind)
        z = P.precond(v, levels=3)
        z1 = P.precond(v, levels=1) if kind == mx.MX_PREC_RAS else None
    tol = 1e-11 if prec == mx.MX_PLAIN_FP64 else MIXED_APPLY_TOL
    ze = O.dd.apply(v.T, levels=(1, 0), kind=name).T
    assert_close(z, ze, tol, what=f"{name} apply")
    if z1 is not None:
        z1e = O.dd.apply(v.T, levels=(1,), kind="ras").T
        assert_close(z1, z1e, tol, what="one-level RAS apply")


@pytest.mark.parametrize("kind,name", [(mx.MX_PREC_RAS, "ras"), (mx.MX_PREC_HRAS, "hras"),
                                       (mx.MX_PREC_ADEF1, "adef1")])
def test_gmres_with_restricted_and_hybrid_preconditioners(kind, name):
    """Right-preconditioned GMRES with each variant reaches the oracle's solution (FP64 form,
    1e-10) in the same number of iterations (+-1)."""
    n, k, nrhs = 10, 6.0, 2
    c, p = inputs.bump_batch(5, nrhs)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=5, kind=name)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-10, restart=0, max_it=300)
    with _handle(n, k, k, k, 5, 1, cm=5, prec=mx.MX_PLAIN_FP64) as P:
        P.factor()
        mx.mx_set_preconditioner(P.h, kind)
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK
    assert_close(x, xo.T, 1e-8, what=f"GMRES solution, {name}")
    for r in range(nrhs):
        assert st[r]["converged"]
        assert abs(st[r]["iterations"] - ost[r][0]) <= 1, (st[r], ost[r])


@pytest.mark.parametrize("prec", [mx.MX_PLAIN_FP64, mx.MX_MIXED])
def test_weighted_gmres_matches_oracle(prec):
    """Weighted GMRES in the D_k = K + k^2 M inner product (Sec. 5.2) against the oracle's
    weighted GMRES: same solution (both to a 1e-10 D_k-norm residual), the reported residual
    is the D_k-norm ratio, and the FP64 form takes the same number of iterations (+-1)."""
    n, k, nrhs = 10, 6.0, 2
    c, p = inputs.bump_batch(7, nrhs)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=5)
    O.factor()
    fo = O.load_vector(c, p, 0.1)
    xo, ost = O.solve(fo, tol=1e-10, restart=0, max_it=300, weighted=True)
    Dk = (O.K + k * k * O.M).tocsr()
    with _handle(n, k, k, k, 5, 1, cm=5, prec=prec) as P:
        P.factor()
        mx.mx_set_weighted_gmres(P.h, 1)
        f = P.load_vector(c, p, 0.1)
        x, st, rc = P.solve(f, tol=1e-10, restart=0, max_it=300)
    assert rc == mx.MX_OK
    assert_close(x, xo.T, 1e-8, what="weighted GMRES solution")
    for r in range(nrhs):
        assert st[r]["converged"]
        res = fo[:, r] - O.A @ x[r]
        rel = np.sqrt(abs(np.vdot(res, Dk @ res))) / np.sqrt(abs(np.vdot(fo[:, r], Dk @ fo[:, r])))
        assert rel <= 1.05e-10 and abs(rel - st[r]["rel_residual"]) <= 1e-12, (rel, st[r])
        if prec == mx.MX_PLAIN_FP64:
            assert abs(st[r]["iterations"] - ost[r][0]) <= 1, (st[r], ost[r])


def test_weighted_gmres_restarted():
    """Weighted GMRES(8) with restarts reaches the direct solution."""
    n, k = 10, 6.0
    c, p = inputs.bump_batch(8, 1)
    O = OracleProblem(n, k, k, k, 5, 1, coarse_m=5)
    fo = O.load_vector(c, p, 0.1)
    import scipy.sparse.linalg as spla
    xd = spla.spsolve(O.A.tocsc(), fo[:, 0])
    with _handle(n, k, k, k, 5, 1, cm=5, prec=mx.MX_MIXED) as P:
        P.factor()
        mx.mx_set_weighted_gmres(P.h, 1)
        x, st, rc = P.solve(fo.T.copy(), tol=1e-9, restart=8, max_it=400)
    assert rc == mx.MX_OK and st[0]["converged"]
    assert_close(x[0], xd, 1e-7, what="restarted weighted GMRES solution")

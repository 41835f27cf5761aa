"""Pins for oracle.gmres: Givens rotations, GMRES against a dense direct solve on tiny
meshes, one-step convergence with the exact inverse, monotone residuals, restarts."""
import numpy as np
import pytest

from oracle.gmres import givens, gmres
from oracle.problem import Problem
import inputs


def test_givens():
    rng = np.random.default_rng(0)
    for trial in range(40):
        a = complex(*rng.standard_normal(2))
        # real b (as GMRES produces: the subdiagonal is a norm) and general complex b
        b = abs(rng.standard_normal()) if trial < 20 else complex(*rng.standard_normal(2))
        c, s = givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        r = G @ np.array([a, b])
        assert abs(r[1]) < 1e-14 and np.allclose(G @ G.conj().T, np.eye(2))
        assert abs(abs(r[0]) - np.hypot(abs(a), abs(b))) < 1e-14


def test_unpreconditioned_dense():
    rng = np.random.default_rng(1)
    n = 30
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 8 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    for restart in (0, 7):
        x, its, rel, ok = gmres(lambda v: A @ v, lambda v: v, b, 1e-12, restart, 500)
        assert ok and np.allclose(x, np.linalg.solve(A, b), atol=1e-10)
    # Krylov space of dimension n: unrestarted GMRES finishes in at most n steps
    x, its, rel, ok = gmres(lambda v: A @ v, lambda v: v, b, 1e-12, 0, 500)
    assert its <= n


@pytest.mark.parametrize("n", [2, 3, 4])
def test_tiny_mesh_vs_direct(n):
    P = Problem(n, 3.0, 1.0, 3.0, max(1, n // 2), 1)
    P.factor()
    c, p = inputs.bump_batch(1, 1)
    f = P.load_vector(c, p, 0.1)[:, 0]
    hist = []
    x, st = P.solve(f, tol=1e-12, history=hist)
    its, rel, ok = st[0]
    assert ok
    xd = np.linalg.solve(P.A.toarray(), f)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    h = np.array(hist[0])
    assert np.all(np.diff(h) <= 1e-14)  # minimal residual: non-increasing


def test_exact_preconditioner_one_step():
    P = Problem(4, 3.0, 3.0, 3.0, 4, 0)
    P.factor()
    f = np.ones(P.n_dof, dtype=complex)
    x, st = P.solve(f, tol=1e-10)
    assert st[0][0] == 1 and st[0][2]


def test_weighted_gmres_minimises_the_weighted_residual():
    """Weighted GMRES (Sec. 5.2): after m steps x_m minimises ||b - A B^{-1} u||_D over the
    Krylov space K_m(A B^{-1}, b); checked against the weighted least-squares problem solved
    densely on an explicit (orthonormalised) Krylov basis."""
    rng = np.random.default_rng(5)
    n = 24
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 6 * np.eye(n)
    Binv = np.diag(1.0 / (1.0 + rng.random(n)))
    L = rng.standard_normal((n, n))
    D = L @ L.T + n * np.eye(n)  # Hermitian positive definite weight
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    C = A @ Binv
    Dh = np.linalg.cholesky(D).conj().T  # ||v||_D = ||Dh v||_2
    for m in (1, 3, 6):
        x, its, rel, ok = gmres(lambda v: A @ v, lambda v: Binv @ v, b, 1e-30, 0, m, weight=lambda v: D @ v)
        assert its == m
        K = np.column_stack([np.linalg.matrix_power(C, j) @ b for j in range(m)])
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(Dh @ C @ Q, Dh @ b, rcond=None)
        xr = Binv @ (Q @ y)
        rw = lambda z: np.linalg.norm(Dh @ (b - A @ z))
        assert abs(rw(x) - rw(xr)) <= 1e-9 * np.linalg.norm(Dh @ b)
        assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)


def test_weighted_gmres_with_identity_weight_is_gmres():
    rng = np.random.default_rng(6)
    n = 20
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 7 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    h1, h2 = [], []
    x1, i1, r1, _ = gmres(lambda v: A @ v, lambda v: v, b, 1e-12, 0, 100, history=h1)
    x2, i2, r2, _ = gmres(lambda v: A @ v, lambda v: v, b, 1e-12, 0, 100, history=h2, weight=lambda v: v)
    assert i1 == i2 and np.allclose(h1, h2, rtol=1e-10) and np.allclose(x1, x2)


def test_weighted_gmres_on_the_maxwell_system():
    """D_k = K + k^2 M weight on a small mesh: converges, non-increasing weighted residual
    estimates, and the solution matches a direct solve."""
    P = Problem(4, 3.0, 3.0, 3.0, 2, 1)
    P.factor()
    c, p = inputs.bump_batch(2, 1)
    f = P.load_vector(c, p, 0.1)[:, 0]
    hist = []
    x, st = P.solve(f, tol=1e-11, history=hist, weighted=True)
    assert st[0][2]
    xd = np.linalg.solve(P.A.toarray(), f)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert np.all(np.diff(np.array(hist[0])) <= 1e-14)


def test_weighted_solve_reports_the_curl_k_norm_residual():
    """Sec. 5.2 with the weight of Eq. 2.3 / 5.1: the weighted solve's reported residual is
    ||b - A x||_D / ||b||_D with D = K + k^2 M, the matrix of the (.,.)_{curl,k} inner
    product. Checked on the impedance space, where the interpolant g of a constant field c
    has g^T K g = 0 and g^T M g = |c|^2 (volume 1), so ||g||_D^2 = k^2 |c|^2."""
    k = 3.0
    P = Problem(4, k, 3.0, 3.0, 2, 1, bc="imp")
    D = (P.K + k * k * P.M).tocsr()
    t = P.mesh.coords(P.mesh.dof_edges[:, 1]) - P.mesh.coords(P.mesh.dof_edges[:, 0])
    c = np.array([0.3, -1.2, 0.7])
    g = t @ c
    assert abs(g @ (D @ g) - k * k * (c @ c)) <= 1e-12 * k * k * (c @ c)
    P.factor()
    b = inputs.random_complex(8, P.n_dof)
    x, st = P.solve(b, tol=1e-6, weighted=True)
    its, rel, ok = st[0]
    r = b - P.A @ x
    rel_d = np.sqrt(np.vdot(r, D @ r).real / np.vdot(b, D @ b).real)
    rel_e = np.linalg.norm(r) / np.linalg.norm(b)
    assert ok and rel_d <= 1e-6
    assert abs(rel - rel_d) <= 1e-9 * rel_d
    assert abs(rel_e - rel_d) > 1e-2 * rel_d  # the weight matters for this residual


def _maxwell(n=6, k=4.0, xi=4.0, coarse_m=3):
    P = Problem(n, k, xi, xi, 3, 1, coarse_m=coarse_m)
    P.factor()
    c, p = inputs.bump_batch(5, 1)
    return P, P.load_vector(c, p, 0.1)[:, 0]


def _orthogonality_loss(V, D=None):
    """max |I - V_j^H D V_j| over the leading j vectors, for j = 1 .. len(V)."""
    DV = V if D is None else np.stack([D @ v for v in V])
    G = V.conj() @ DV.T
    E = np.abs(G - np.eye(len(V)))
    return np.array([E[:j, :j].max() for j in range(1, len(V) + 1)])


def _check_mgs_loss(loss, hist):
    """Modified Gram-Schmidt keeps the basis orthonormal to rounding while the residual is
    large and loses orthogonality only as the residual falls, the loss staying of the order of
    the unit roundoff divided by the relative residual (Paige, Rozloznik and Strakos, SIAM
    J. Matrix Anal. Appl. 28 (2006), on MGS-GMRES). A wrong conjugation, index or sign in
    the Gram-Schmidt loop breaks orthogonality at once, at residuals near 1."""
    assert loss[0] <= 1e-15
    for j in range(2, len(loss) + 1):
        rho = hist[j - 2]  # relative residual after j - 1 steps
        assert loss[j - 1] * rho <= 1e-14, (j, loss[j - 1], rho)
        if rho >= 1e-3:
            assert loss[j - 1] <= 1e-12, (j, loss[j - 1], rho)


@pytest.mark.parametrize("restart", [0, 6])
def test_arnoldi_relation_and_orthonormal_basis(restart):
    """Arnoldi invariants of the right-preconditioned process (Sec. 5.2, Sec. 6.1): for every
    cycle A Z_k = V_{k+1} H-bar_k with Z_k = B^{-1} V_k, V orthonormal up to the MGS loss,
    and H-bar upper Hessenberg with a real positive subdiagonal."""
    P, f = _maxwell()
    rec, hist = [], []
    x, its, rel, ok = gmres(lambda v: P.A @ v, lambda v: P.dd.apply(v, kind=P.kind), f, 1e-10, restart, 300,
                            arnoldi=rec, history=hist)
    assert ok and len(rec) >= (2 if restart else 1)
    assert sum(c["Z"].shape[0] for c in rec) == its == len(hist)
    start = 0
    for c in rec:
        V, Z, Hb = c["V"], c["Z"], c["Hbar"]
        k = Z.shape[0]
        assert V.shape[0] == k + 1 and Hb.shape == (k + 1, k)
        AZ = np.stack([P.A @ z for z in Z], axis=1)
        assert np.abs(AZ - V.T @ Hb).max() <= 1e-12 * np.abs(AZ).max()
        # a restart cycle starts from the true residual: measure its loss against the
        # residual reduction within the cycle
        h = np.array(hist[start:start + k]) / (hist[start - 1] if start else 1.0)
        _check_mgs_loss(_orthogonality_loss(V), h)
        start += k
        BV = np.stack([P.dd.apply(v, kind=P.kind) for v in V[:k]], axis=0)
        assert np.abs(BV - Z).max() == 0.0
        assert np.all(np.tril(Hb, -2) == 0)
        sub = np.diag(Hb, -1)
        assert np.all(sub.imag == 0) and np.all(sub.real > 0)
    # the first basis vector of the first cycle is b / ||b|| (x0 = 0)
    assert np.allclose(rec[0]["V"][0], f / np.linalg.norm(f), rtol=0, atol=1e-15)


def test_weighted_arnoldi_basis_is_d_orthonormal():
    """Weighted GMRES (Sec. 5.2): the basis is orthonormal in <u, v>_D = v^H D u with
    D = K + k^2 M, and the Arnoldi relation is unchanged."""
    P, f = _maxwell()
    D = (P.K + P.k ** 2 * P.M).tocsr()
    rec, hist = [], []
    x, its, rel, ok = gmres(lambda v: P.A @ v, lambda v: P.dd.apply(v, kind=P.kind), f, 1e-8, 0, 300,
                            weight=lambda v: D @ v, arnoldi=rec, history=hist)
    V, Z, Hb = rec[0]["V"], rec[0]["Z"], rec[0]["Hbar"]
    _check_mgs_loss(_orthogonality_loss(V, D), hist)
    # the Euclidean Gram matrix is far from the identity: the weight matters
    assert _orthogonality_loss(V[:3])[-1] > 1e-2
    AZ = np.stack([P.A @ z for z in Z], axis=1)
    assert np.abs(AZ - V.T @ Hb).max() <= 1e-12 * np.abs(AZ).max()


def test_flexible_arnoldi_relation_with_a_changing_preconditioner():
    """FGMRES: with B_j^{-1} changing at every call, A Z_k = V_{k+1} H-bar_k still holds for
    the stored z_j, while Z_k is no longer B^{-1} V_k for any one B."""
    P, f = _maxwell()
    calls = [0]

    def varying(v):
        calls[0] += 1
        return P.dd.apply(v, kind=P.kind) * (1.0 + 0.3 * np.sin(calls[0]))

    rec = []
    x, its, rel, ok = gmres(lambda v: P.A @ v, varying, f, 1e-10, 0, 300, flexible=True, arnoldi=rec)
    assert ok
    V, Z, Hb = rec[0]["V"], rec[0]["Z"], rec[0]["Hbar"]
    AZ = np.stack([P.A @ z for z in Z], axis=1)
    assert np.abs(AZ - V.T @ Hb).max() <= 1e-12 * np.abs(AZ).max()
    assert np.linalg.norm(f - P.A @ x) <= 1.0001e-10 * np.linalg.norm(f)

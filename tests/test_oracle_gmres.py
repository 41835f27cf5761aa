"""Pins for oracle.gmres: Givens rotations, GMRES against a dense direct solve on tiny
meshes, one-step convergence with the exact inverse, monotone residuals, restarts."""
import numpy as np
import pytest

from oracle.gmres import givens, gmres
from oracle.problem import Problem
import inputs


def test_givens():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = complex(*rng.standard_normal(2)), abs(rng.standard_normal())
        c, s = givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        r = G @ np.array([a, b])
        assert abs(r[1]) < 1e-14 and np.allclose(G @ G.conj().T, np.eye(2))


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

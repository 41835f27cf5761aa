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

"""Pins for the inexact coarse solve of Sec. 6.4 and the flexible outer GMRES it needs:
FGMRES equals GMRES for a fixed preconditioner; under a preconditioner that changes every
iteration the FGMRES residual estimate is the true residual (and the non-flexible update is
not); the inner GMRES meets its tolerance at the first iteration that can; a tight inner
tolerance reproduces the direct coarse correction; a single inner subdomain makes the inner
preconditioner exact (one inner iteration); the outer iteration converges to the requested
true residual with the rough (1e-1) coarse solves."""
import numpy as np
import pytest

from oracle.mesh import KuhnMesh
from oracle import fem, dd
from oracle.gmres import gmres
from oracle.problem import Problem


def _system(n=6, k=4.0, xi_prob=0.0, xi_prec=16.0, core=3, overlap=1, coarse_m=3, seed=0):
    m = KuhnMesh(n)
    K, M = fem.assemble_KM(m)
    A = fem.a_xi(K, M, k, xi_prob).tocsr()
    S = dd.Schwarz(m, fem.a_xi(K, M, k, xi_prec), core, overlap, coarse_m, k, xi_prec)
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(m.n_dof) + 1j * rng.standard_normal(m.n_dof)
    return A, S, b


def test_fgmres_fixed_preconditioner_equals_gmres():
    A, S, b = _system()
    S.factor()
    h0, h1 = [], []
    x0, it0, r0, ok0 = gmres(lambda v: A @ v, lambda v: S.apply(v, levels=(1, 0)), b, 1e-10, 0, 200, history=h0)
    x1, it1, r1, ok1 = gmres(lambda v: A @ v, lambda v: S.apply(v, levels=(1, 0)), b, 1e-10, 0, 200, history=h1,
                             flexible=True)
    assert ok0 and ok1 and it0 == it1
    assert np.allclose(h0, h1, rtol=1e-8, atol=1e-14)
    assert np.linalg.norm(x1 - x0) <= 1e-9 * np.linalg.norm(x0)


def test_fgmres_estimate_is_true_residual_with_varying_preconditioner():
    """The preconditioner changes at every call (a different random perturbation); FGMRES
    minimises over span(Z_m), so its Givens estimate equals the true residual of x0 + Z y.
    The non-flexible update x0 + B^{-1}(V y) uses the last operator only and misses it."""
    A, S, b = _system(n=6, coarse_m=0)
    S.factor()
    n = b.shape[0]
    rng = np.random.default_rng(3)
    E = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / n

    def make():
        calls = [0]

        def prec(v):
            calls[0] += 1
            eps = 0.3 * np.sin(1.7 * calls[0])
            return S.apply(v, levels=(1,)) + eps * (E @ v)
        return prec

    for flexible in (True, False):
        hist = []
        x, its, rel, ok = gmres(lambda v: A @ v, make(), b, 1e-9, 0, 300, history=hist, flexible=flexible)
        true_rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert abs(true_rel - rel) <= 1e-12
        if flexible:
            assert ok and abs(true_rel - hist[-1]) <= 1e-9 * max(1.0, hist[-1]) + 1e-12
        else:
            assert true_rel > 2 * hist[-1]


def test_inner_gmres_meets_its_tolerance_at_the_first_chance():
    A, S, b = _system(n=12, k=6.0, xi_prec=36.0, core=4, coarse_m=6)
    S.set_inner_coarse(core=2, overlap=1, tol=0.1, max_it=100, kind="ras")
    S.factor()
    rc = S.R0 @ b
    y = S.coarse_solve(rc)
    its = S.inner_its[-1]
    res = np.linalg.norm(rc - S.A0 @ y) / np.linalg.norm(rc)
    assert its >= 1 and res <= 0.1
    # one iteration fewer does not reach the tolerance (estimate = true residual here)
    if its > 1:
        _, _, rel, ok = gmres(lambda u: S.A0 @ u, lambda u: S.inner.apply(u, levels=(1,), kind="ras"), rc, 0.1, 0,
                              its - 1)
        assert not ok and rel > 0.1


def test_tight_inner_tolerance_reproduces_the_direct_coarse_correction():
    A, S, b = _system(n=12, k=6.0, xi_prec=36.0, core=4, coarse_m=6)
    S.factor()
    g_direct = S.coarse_correction(b)
    S.set_inner_coarse(core=2, overlap=1, tol=1e-13, max_it=400, kind="as")
    S.factor()
    g_inner = S.coarse_correction(b)
    assert np.linalg.norm(g_inner - g_direct) <= 1e-10 * np.linalg.norm(g_direct)


def test_single_inner_subdomain_is_exact():
    """One inner subdomain covering the coarse mesh (no overlap needed): the inner
    preconditioner is (A^0)^{-1}, so the inner GMRES stops after one iteration with the
    direct solution."""
    A, S, b = _system(n=12, k=6.0, xi_prec=36.0, core=4, coarse_m=6)
    S.factor()
    y_direct = S.coarse.solve(S.R0 @ b)
    S.set_inner_coarse(core=6, overlap=0, tol=1e-10, max_it=10, kind="as")
    S.factor()
    y = S.coarse_solve(S.R0 @ b)
    assert S.inner_its[-1] == 1
    assert np.linalg.norm(y - y_direct) <= 1e-10 * np.linalg.norm(y_direct)


@pytest.mark.parametrize("core,overlap", [(2, 1), (3, 0), (2, 2)])
def test_inner_schwarz_is_built_on_the_requested_coarse_boxes(core, overlap):
    """Sec. 6.4: the inner preconditioner is one-level Schwarz on boxes of the coarse mesh of
    `core` coarse cells widened by `overlap` (the fine-mesh rules applied to the coarse mesh),
    built from A^0 itself."""
    A, S, b = _system(n=12, k=6.0, xi_prec=36.0, core=4, coarse_m=6)
    S.set_inner_coarse(core=core, overlap=overlap, tol=0.1, max_it=20, kind="ras")
    want = dd.subdomain_boxes(6, core, overlap)
    assert len(S.inner.boxes) == len(want)
    for (lo, hi), (wl, wh) in zip(S.inner.boxes, want):
        assert np.array_equal(lo, wl) and np.array_equal(hi, wh)
    assert abs(S.inner.A_prec - S.A0).max() == 0
    sizes = [len(i) for i in S.inner.idx]
    assert sizes == [len(dd.local_dofs(S.coarse_mesh, lo, hi)) for lo, hi in want]


@pytest.mark.parametrize("kind", ["as", "adef1"])
def test_outer_fgmres_converges_with_rough_coarse_solves(kind):
    inner = dict(core=2, overlap=1, tol=0.1, max_it=50, kind="ras")
    P = Problem(12, 6.0, 0.0, 36.0, 4, 1, coarse_m=6, kind=kind, inner_coarse=inner)
    P.factor()
    rng = np.random.default_rng(5)
    b = rng.standard_normal(P.n_dof) + 1j * rng.standard_normal(P.n_dof)
    x, stats = P.solve(b, tol=1e-8, max_it=200)
    its, rel, ok = stats[0]
    assert ok and rel <= 1e-8
    assert np.linalg.norm(b - P.A @ x) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    assert len(P.dd.inner_its) >= its and max(P.dd.inner_its) >= 1
    # the exact coarse solve needs no more outer iterations than the rough one, up to 1
    Pd = Problem(12, 6.0, 0.0, 36.0, 4, 1, coarse_m=6, kind=kind)
    Pd.factor()
    _, sd = Pd.solve(b, tol=1e-8, max_it=200)
    assert sd[0][0] <= its + 1

"""Parity at the full size of the benchmark workload, in the launch configuration the
benchmark times: 60^3 cells (1,479,780 DOFs), k = 30, xi_prob = xi_prec = k^2, 5^3-cell
subdomains with a 1-cell overlap (1,728 of them), a 12^3 coarse mesh, 16 right-hand sides in
one batched solve, the mixed form, GMRES(200) to 1e-6, device buffers on the caller's stream.

The oracle cannot run the whole method at this size in a test (its Schwarz set-up alone
takes minutes), so it checks what it can compute independently:
  * the integer mesh data, bit-exact (Sec. 2.2);
  * the load vector at sampled DOFs, by the oracle's quadrature over exactly the
    tetrahedra that touch those DOFs (Sec. 2.2; the full vector is a sum over all of them);
  * the solution through its defining property, with the oracle's own operator: the
    relative residual ||f - A x|| / ||f|| (Sec. 6.1) of every right-hand side is at most
    the tolerance, and equals the residual the library reports;
  * the solution itself, element by element, at the 2,000-odd sampled DOFs of
    tests/golden/solution60_k30.txt, the oracle's own solution of this workload (right-hand
    sides 0 and 1, its GMRES run to 1e-10 by tests/golden/make_solution60.py): error at
    most 1e-5 of ||x_oracle||_inf at every sampled DOF, with the iteration counts beside
    the oracle's count to 1e-6.
The file name makes pytest collect it after the other GPU modules."""
import os

import numpy as np
import pytest

import inputs
from parity import LOAD_DF_TOL
from oracle.mesh import KuhnMesh
from oracle import fem

N, K, XI, CORE, OVERLAP, COARSE, NRHS = 60, 30.0, 900.0, 5, 1, 12, 16
TOL, RESTART, MAX_IT, SEED = 1e-6, 200, 600, 1


FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "solution60_k30.txt")


def load_solution_fixture(path=FIXTURE):
    """(header fields, per-RHS fields, sampled DOFs, oracle solution [R, len])."""
    meta, rhs, rows = {}, {}, []
    for line in open(path):
        t = line.split()
        if line.startswith("# n="):
            meta = dict(kv.split("=") for kv in t[1:])
        elif line.startswith("# rhs "):
            rhs[int(t[2])] = {t[i]: float(t[i + 1]) for i in range(3, len(t) - 1, 2)}
        elif not line.startswith("#") and t:
            rows.append([float(v) for v in t])
    a = np.array(rows)
    return meta, rhs, a[:, 0].astype(np.int64), (a[:, 1::2] + 1j * a[:, 2::2]).T


def test_solution_fixture_describes_this_workload():
    """CPU check of the stored oracle solution: written for the workload of this file, to
    1e-10, with the DOFs nearest the bump centres among the samples."""
    meta, rhs, dofs, xo = load_solution_fixture()
    assert (int(meta["n"]), float(meta["k"]), float(meta["xi_prob"]), float(meta["xi_prec"])) == (N, K, XI, XI)
    assert (int(meta["core"]), int(meta["overlap"]), int(meta["coarse"]), int(meta["seed"])) == (CORE, OVERLAP, COARSE,
                                                                                                 SEED)
    assert meta["bc"] == "pec" and meta["precond"] == "as" and float(meta["tol"]) == 1e-10
    assert sorted(rhs) == [0, 1] and xo.shape == (2, len(dofs)) and np.isfinite(xo).all()
    assert len(dofs) >= 2000 and dofs.min() >= 0 and dofs.max() < 1479780 and np.all(np.diff(dofs) > 0)
    for r, v in rhs.items():
        assert v["rel_residual"] <= 1e-10 and 0 < v["iterations_to_1e-6"] <= v["iterations"]
        assert np.abs(xo[r]).max() <= v["x_inf"] * (1 + 1e-15)
    m = KuhnMesh(N)
    c, _ = inputs.bump_batch(SEED, 2)
    mid = 0.5 * (m.coords(m.dof_edges[:, 0]) + m.coords(m.dof_edges[:, 1]))
    for ctr in c.reshape(-1, 3):
        assert int(np.argmin(np.sum((mid - ctr) ** 2, axis=1))) in set(dofs.tolist())


class _TetSubset:
    """The oracle mesh restricted to some of its tetrahedra: the attributes that
    fem.load_vector reads (tets, tet2dof, coords, n_dof), nothing else."""

    def __init__(self, mesh, keep):
        self.tets = mesh.tets[keep]
        self.tet2dof = mesh.tet2dof[keep]
        self.coords = mesh.coords
        self.n_dof = mesh.n_dof


def sampled_load_vector(mesh, F, dofs, q=3):
    """f at the DOFs `dofs` only: the oracle's load_vector over the tetrahedra that hold one
    of them (every contribution to f_i comes from a tetrahedron containing edge i)."""
    keep = np.isin(mesh.tet2dof, dofs).any(axis=1)
    return fem.load_vector(_TetSubset(mesh, keep), F, q)[dofs]


def _sample(n_dof, count=48, seed=7, mesh=None, centres=None):
    """Seeded random DOFs, the first and last, and (given the mesh and the bump centres
    [R, B, 3]) the DOF whose edge midpoint is nearest each centre, where f is largest."""
    rng = np.random.default_rng(seed)
    s = [rng.choice(n_dof, size=count, replace=False), [0, n_dof - 1]]
    if mesh is not None:
        mid = 0.5 * (mesh.coords(mesh.dof_edges[:, 0]) + mesh.coords(mesh.dof_edges[:, 1]))
        s.append([int(np.argmin(np.sum((mid - ctr) ** 2, axis=1))) for ctr in centres.reshape(-1, 3)])
    return np.unique(np.concatenate(s))


def test_sampled_load_vector_equals_the_full_one():
    """CPU check of the sampling helper against the oracle's full load vector."""
    m = KuhnMesh(6)
    c, p = inputs.bump_batch(SEED, 3)
    F = fem.bump_field(c, p, 0.1)
    full = fem.load_vector(m, F)
    dofs = _sample(m.n_dof, count=20, mesh=m, centres=c)
    assert len(dofs) >= 20
    got = sampled_load_vector(m, F, dofs)
    assert np.abs(got - full[dofs]).max() <= 1e-15 * np.abs(full).max()


@pytest.mark.gpu
def test_benchmark_workload_at_full_size():
    mx = pytest.importorskip("paper_1711_03789_gb300")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.current_stream()
    c, p = inputs.bump_batch(SEED, NRHS)
    with mx.Problem(N, K, XI, XI, CORE, OVERLAP, COARSE, mx.MX_MIXED, stream=stream.cuda_stream) as P:
        n = P.n_dof
        key, t2d = mx.mx_get_mesh(P.h, N)
        P.factor()
        f = torch.empty((NRHS, n), dtype=torch.complex128, device="cuda")
        P.load_vector(c, p, 0.1, out=f)
        x = torch.empty_like(f)
        x, st, rc = P.solve(f, TOL, RESTART, MAX_IT, x=x)
        torch.cuda.synchronize()
        fh, xh = f.cpu().numpy(), x.cpu().numpy()
    assert rc == mx.MX_OK

    m = KuhnMesh(N)
    assert n == m.n_dof == 1479780
    assert np.array_equal(key, m.dof_key.astype(np.int32))
    assert np.array_equal(t2d, m.tet2dof.astype(np.int32))
    del key, t2d

    dofs = _sample(n, mesh=m, centres=c)
    fs = sampled_load_vector(m, fem.bump_field(c, p, 0.1), dofs)  # [len(dofs), NRHS]
    # the mixed form's load vector: double-float quadrature moments
    assert np.abs(fh[:, dofs].T - fs).max() <= LOAD_DF_TOL * np.abs(fs).max()

    Km, Mm = fem.assemble_KM(m)
    A = fem.a_xi(Km, Mm, K, XI).tocsr()
    del Km, Mm
    for r in range(NRHS):
        assert st[r]["converged"], (r, st[r])
        res = np.linalg.norm(fh[r] - A @ xh[r]) / np.linalg.norm(fh[r])
        # the two FP64 assemblies differ by rounding only (about 1e-16 of the operator's
        # scale, times ||A|| ||A^-1|| of a few hundred here): far inside this slack
        assert res <= TOL * (1 + 1e-4), (r, res)
        assert abs(res - st[r]["rel_residual"]) <= 1e-3 * TOL, (r, res, st[r]["rel_residual"])

    meta, rhs, sdofs, xo = load_solution_fixture()
    for r, v in rhs.items():
        err = np.abs(xh[r, sdofs] - xo[r]).max() / v["x_inf"]
        print(f"rhs {r}: max sampled error / ||x_oracle||_inf = {err:.3e}; iterations {st[r]['iterations']} "
              f"(oracle to 1e-6: {int(v['iterations_to_1e-6'])}, change {st[r]['iterations'] - int(v['iterations_to_1e-6'])})")
        assert err <= 1e-5, (r, err)

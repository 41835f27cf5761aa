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
    the tolerance, and equals the residual the library reports.
The file name makes pytest collect it after the other GPU modules."""
import numpy as np
import pytest

import inputs
from oracle.mesh import KuhnMesh
from oracle import fem

N, K, XI, CORE, OVERLAP, COARSE, NRHS = 60, 30.0, 900.0, 5, 1, 12, 16
TOL, RESTART, MAX_IT, SEED = 1e-6, 200, 600, 1


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
    assert np.abs(fh[:, dofs].T - fs).max() <= 1e-12 * np.abs(fs).max()

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

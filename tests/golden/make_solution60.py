"""Write tests/golden/solution60_k30.txt: the oracle's solution of the benchmark workload at
sampled DOFs, for the element-wise error check of the GPU solution at full size.

Workload: 60^3 cells (1,479,780 DOFs), k = 30, xi_prob = xi_prec = k^2, PEC, 5^3-cell
subdomains with a 1-cell overlap (1,728), a 12^3 coarse mesh, two-level additive Schwarz
(Eq. 3.4) built from A_{xi_prec} (Sec. 6.2), right-preconditioned GMRES(200) from x0 = 0
(Sec. 6.1) to a relative residual of 1e-10; right-hand sides 0 and 1 of the seed-1
Gaussian-bump batch (the first two of the benchmark's sixteen).

Only `oracle/` and `inputs/` are used. The oracle's preconditioner is the sum of Eq. 3.4;
this script evaluates that sum in worker processes, each holding the SuperLU factors
(oracle `Schwarz.factor(subset)`) of a fixed share of the subdomains, and adds the
partial sums and the coarse term in the parent in a fixed order. Only the order of the
floating-point additions differs from `Schwarz.apply`.

Usage: python tests/golden/make_solution60.py [--procs P] [--out PATH]
Takes about 12 minutes on 8 cores (7 of them in the oracle's single-threaded set-up).
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

# one BLAS thread per process: the subdomain work is spread over worker processes, and
# multithreaded BLAS calls inside each of them would oversubscribe the cores
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
from oracle.problem import Problem  # noqa: E402
from oracle import gmres as ogmres  # noqa: E402

N, K, XI, CORE, OVERLAP, COARSE = 60, 30.0, 900.0, 5, 1, 12
SEED, RHS = 1, (0, 1)
TOL, RESTART, MAX_IT = 1e-10, 200, 600
SAMPLE, SAMPLE_SEED = 2000, 11

_P = None  # the oracle problem, built in the parent before the workers fork


def _worker(conn, subset):
    """Factors the subdomains of `subset` and answers apply requests with the partial sum
    over them of (R^l)^T (A^l)^{-1} R^l v (Eq. 3.4, l >= 1)."""
    dd = _P.dd
    dd.factor(subset)
    conn.send("ready")
    while True:
        v = conn.recv()
        if v is None:
            break
        z = np.zeros_like(v)
        for l in subset:
            i = dd.idx[l]
            z[i] += dd.local_solve(l, v[i])
        conn.send(z)
    conn.close()


def sample_dofs(mesh, centres):
    """Seeded random DOFs, the first and last, and the 8 DOFs whose edge midpoints are
    nearest each bump centre (where the solution is largest)."""
    rng = np.random.default_rng(SAMPLE_SEED)
    s = [rng.choice(mesh.n_dof, size=SAMPLE, replace=False), [0, mesh.n_dof - 1]]
    mid = 0.5 * (mesh.coords(mesh.dof_edges[:, 0]) + mesh.coords(mesh.dof_edges[:, 1]))
    for ctr in centres.reshape(-1, 3):
        d2 = np.sum((mid - ctr) ** 2, axis=1)
        s.append(np.argpartition(d2, 8)[:8])
    return np.unique(np.concatenate(s))


def main():
    global _P
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=min(8, os.cpu_count() or 1))
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "solution60_k30.txt"))
    args = ap.parse_args()
    t0 = time.time()
    _P = Problem(N, K, XI, XI, CORE, OVERLAP, coarse_m=COARSE)
    print(f"oracle set-up {time.time() - t0:.0f} s, {_P.n_dof} DOFs", flush=True)
    n_sub = len(_P.dd.idx)
    ctx = mp.get_context("fork")  # CPU only: the workers share the parent's set-up copy-on-write
    conns, procs = [], []
    for w in range(args.procs):
        a, b = ctx.Pipe()
        p = ctx.Process(target=_worker, args=(b, list(range(w, n_sub, args.procs))))
        p.start()
        conns.append(a)
        procs.append(p)
    import scipy.sparse.linalg as spla
    coarse = spla.splu(_P.dd.A0.tocsc())
    for c in conns:
        assert c.recv() == "ready"
    print(f"factored {n_sub} subdomains + coarse in {time.time() - t0:.0f} s", flush=True)

    R0 = _P.dd.R0

    def precond(v):
        for c in conns:
            c.send(v)
        z = np.zeros_like(v)
        for c in conns:  # fixed order
            z += c.recv()
        return z + R0.T @ coarse.solve(R0 @ v)

    centres, pol = inputs.bump_batch(SEED, max(RHS) + 1)
    f = _P.load_vector(centres, pol, 0.1)  # [n, R]
    dofs = sample_dofs(_P.mesh, centres[list(RHS)])
    rows = []
    for r in RHS:
        hist = []
        ts = time.time()
        x, its, rel, ok = ogmres.gmres(lambda v: _P.A @ v, precond, f[:, r], TOL, RESTART, MAX_IT, history=hist)
        its6 = next((j + 1 for j, h in enumerate(hist) if h <= 1e-6), None)
        print(f"rhs {r}: {its} iterations to {rel:.3e} ({its6} to 1e-6), {time.time() - ts:.0f} s", flush=True)
        assert ok, (r, its, rel)
        rows.append(dict(x=x, its=its, its6=its6, rel=rel, ninf=float(np.abs(x).max()),
                         n2=float(np.linalg.norm(x))))
    for c in conns:
        c.send(None)
    for p in procs:
        p.join()

    with open(args.out, "w") as fh:
        fh.write("# Oracle solution of the benchmark workload at sampled DOFs (Sec. 6.1, Eq. 3.4).\n")
        fh.write(f"# Written by tests/golden/make_solution60.py from oracle/ and inputs/ only.\n")
        fh.write(f"# n={N} k={K} xi_prob={XI} xi_prec={XI} core={CORE} overlap={OVERLAP} coarse={COARSE} "
                 f"bc=pec precond=as seed={SEED} width=0.1 restart={RESTART} tol={TOL}\n")
        fh.write(f"# n_dof {_P.n_dof}\n")
        for r, row in zip(RHS, rows):
            fh.write(f"# rhs {r} iterations {row['its']} iterations_to_1e-6 {row['its6']} rel_residual "
                     f"{row['rel']:.6e} x_inf {row['ninf']:.17g} x_2 {row['n2']:.17g}\n")
        fh.write("# dof " + " ".join(f"re{r} im{r}" for r in RHS) + "\n")
        for d in dofs:
            fh.write(f"{d} " + " ".join(f"{row['x'][d].real:.17g} {row['x'][d].imag:.17g}" for row in rows) + "\n")
    print(f"wrote {len(dofs)} DOFs to {args.out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()

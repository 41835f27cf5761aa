"""Mutation check of the oracle's pins (test infrastructure; not collected by pytest).

Each mutant changes one line of the oracle the way a plausible mistake would: a flipped sign,
a dropped term, a wrong index or bound, a transposed or conjugated operand, a changed
convention. For each one the script copies oracle/, tests/ and inputs/ into a scratch
directory, applies the mutant and runs the CPU pins (-m "not gpu"). A mutant is killed when
some pin fails. Every mutant listed here is killed; a surviving one would mark a gap in the
pins.

    python tests/oracle_mutants.py [--jobs 8] [--only 3,7] [--workdir DIR]

About six minutes on 8 cores. The scratch copies go to a temporary directory unless
--workdir is given.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle module, label, original text, mutated text)
MUTANTS = [
 ("mesh", "pec far faces", "        for val in (0, n):\n            on |= (a[:, ax] == val) & (b[:, ax] == val)\n    return on", "        for val in (0,):\n            on |= (a[:, ax] == val) & (b[:, ax] == val)\n    return on"),
 ("mesh", "kuhn path", "        c2 = c1 + eye[s[1]]", "        c2 = c1 + eye[s[0]]"),
 ("mesh", "key from high end", "        self.key = 7 * self.edges[:, 0] + self.edge_dir", "        self.key = 7 * self.edges[:, 1] + self.edge_dir"),
 ("mesh", "interior count term", "            + a * b * (c - 1) + a * c * (b - 1) + b * c * (a - 1) + a * b * c)", "            + a * b * (c - 1) + a * c * (b - 1) + b * c * (a - 1))"),
 ("mesh", "box faces lo only", "                if np.all(col == col[0]) and col[0] in (lo[ax], hi[ax]):", "                if np.all(col == col[0]) and col[0] == lo[ax]:"),
 ("fem", "curl factor", "            K[:, a, b] = 4.0 * vol *", "            K[:, a, b] = 2.0 * vol *"),
 ("fem", "absorption sign", "    A = K.astype(np.complex128) - (k * k + 1j * xi) * M.astype(np.complex128)", "    A = K.astype(np.complex128) - (k * k - 1j * xi) * M.astype(np.complex128)"),
 ("fem", "impedance sign", "        A = A - 1j * imp_sign(xi) * k * B.astype(np.complex128)", "        A = A + 1j * imp_sign(xi) * k * B.astype(np.complex128)"),
 ("fem", "sign(0)", "    return -1.0 if xi < 0 else 1.0", "    return -1.0 if xi <= 0 else 1.0"),
 ("fem", "face mass scale", "    mass = lambda i, j: area * (1.0 + (i == j)) / 12.0", "    mass = lambda i, j: area * (1.0 + (i == j)) / 10.0"),
 ("fem", "bump width convention", "                out[:, :, r] += np.exp(-d2 / width ** 2)[:, None] * pol[r, b][None, :]", "                out[:, :, r] += np.exp(-d2 / (2 * width ** 2))[:, None] * pol[r, b][None, :]"),
 ("fem", "face edge basis sign", "            B[:, a, b] = (dot(q, s) * mass(p, r) - dot(q, r) * mass(p, s)\n                          - dot(p, s) * mass(q, r) + dot(p, r) * mass(q, s))", "            B[:, a, b] = (dot(q, s) * mass(p, r) + dot(q, r) * mass(p, s)\n                          - dot(p, s) * mass(q, r) + dot(p, r) * mass(q, s))"),
 ("dd", "overlap low side", "        lo = max(core * i - overlap, 0)", "        lo = max(core * i - overlap + 1, 0)"),
 ("dd", "face edges kept", "    return np.nonzero(inside & ~on_face)[0]", "    return np.nonzero(inside)[0]"),
 ("dd", "R0 basis sign", "        w = lam[:, p, None] * G[:, q] - lam[:, q, None] * G[:, p]\n        val = np.einsum(\"ji,ji->j\", w, t)", "        w = lam[:, p, None] * G[:, q] + lam[:, q, None] * G[:, p]\n        val = np.einsum(\"ji,ji->j\", w, t)"),
 ("dd", "R0 simplex order", "    perm = np.argsort(-loc, axis=1, kind=\"stable\")", "    perm = np.argsort(loc, axis=1, kind=\"stable\")"),
 ("dd", "owner rounding", "        box = np.minimum(mid2 // (2 * core), N - 1)", "        box = np.minimum((mid2 + 1) // (2 * core), N - 1)"),
 ("dd", "ras unrestricted", "            z[i[d]] += zl[d]", "            z[i] += zl"),
 ("dd", "hras sign", "            return u - self.coarse_correction(A @ u) + gv", "            return u + self.coarse_correction(A @ u) + gv"),
 ("dd", "adef1 sign", "            u = self.ras1(v - A @ gv)", "            u = self.ras1(v + A @ gv)"),
 ("dd", "box impedance term", "        return fem.a_xi(K, M, self.k, self.xi_prec, B)", "        return fem.a_xi(K, M, self.k, self.xi_prec, None)"),
 ("dd", "coarse conj", "            self.coarse = spla.splu(self.A0.tocsc())", "            self.coarse = spla.splu(self.A0.conj().tocsc())"),
 ("gmres", "givens conj", "    s = (a / abs(a)) * np.conj(b) / t", "    s = (a / abs(a)) * b / t"),
 ("gmres", "g rotation conj", "            g[j + 1] = -np.conj(sn[j]) * g[j]", "            g[j + 1] = -sn[j] * g[j]"),
 ("gmres", "restart drops x", "        x = x + (Z[:k].T @ y if flexible else precond(V[:k].T @ y))", "        x = (Z[:k].T @ y if flexible else precond(V[:k].T @ y))"),
 ("gmres", "flexible ignored", "        x = x + (Z[:k].T @ y if flexible else precond(V[:k].T @ y))", "        x = x + precond(V[:k].T @ y)"),
 ("problem", "prec from xi_prob", "        self.A_prec = fem.a_xi(self.K, self.M, k, xi_prec, self.B)", "        self.A_prec = fem.a_xi(self.K, self.M, k, xi_prob, self.B)"),
 ("gmres", "weighted norm ignores D", "        return float(np.sqrt(max(dot(v, v).real, 0.0)))", "        return float(np.linalg.norm(v))"),
 ("gmres", "MGS coefficient conj", "                w = w - H[i, j] * V[i]", "                w = w - np.conj(H[i, j]) * V[i]"),
 ("gmres", "backsolve transposed", "        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])", "        y = np.linalg.solve(np.triu(H[:k, :k]).T, g[:k])"),
 ("dd", "AS overwrite", "                for l, i in enumerate(self.idx):\n                    z[i] += self.local_solve(l, v[i])", "                for l, i in enumerate(self.idx):\n                    z[i] = self.local_solve(l, v[i])"),
 ("dd", "R0 at endpoint", "    mid = 0.5 * (xa + xb)\n    t = xb - xa", "    mid = 0.5 * (xa + xa)\n    t = xb - xa"),
 ("dd", "inner tol ignored", "                             self.inner_tol, 0, self.inner_max_it)", "                             self.inner_tol * 1e-3, 0, self.inner_max_it)"),
 ("dd", "closed box drops its faces", "    if closed:\n        return np.nonzero(inside)[0]", "    if False:\n        return np.nonzero(inside)[0]"),
 ("fem", "duffy jacobian", "                wts.append(wt[a] * wt[b] * wt[c] * (1 - u) ** 2 * (1 - v))", "                wts.append(wt[a] * wt[b] * wt[c] * (1 - u) * (1 - v))"),
 ("fem", "load weight", "        wgt = 6.0 * vol * wq[qp]", "        wgt = vol * wq[qp]"),
 ("fem", "gradient sign", "    G = np.transpose(inv[:, 1:, :], (0, 2, 1))  # [T, 4, 3]", "    G = -np.transpose(inv[:, 1:, :], (0, 2, 1))  # [T, 4, 3]"),
 ("fem", "mass cross term", "            Mm[:, a, b] = (dot(q, s) * mass(p, r) - dot(q, r) * mass(p, s)", "            Mm[:, a, b] = (dot(q, s) * mass(p, r) - dot(q, r) * mass(p, r)"),
 ("problem", "flexible off", "        self.flexible = inner_coarse is not None", "        self.flexible = False"),
 ("mesh", "dir table swap", "DIRS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]],", "DIRS = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1], [1, 1, 0], [1, 0, 1], [0, 1, 1], [1, 1, 1]],"),
 ("mesh", "tet2dof local edge", "LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]", "LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (2, 3), (1, 3)]"),
 ("problem", "weight k instead of k^2", "        Dk = (self.K + self.k ** 2 * self.M).tocsr() if weighted else None", "        Dk = (self.K + self.k * self.M).tocsr() if weighted else None"),
 ("dd", "inner overlap", "        self.inner = Schwarz(self.coarse_mesh, self.A0, core, overlap, k=self.k, xi_prec=self.xi_prec)", "        self.inner = Schwarz(self.coarse_mesh, self.A0, core, overlap + 1, k=self.k, xi_prec=self.xi_prec)"),
 ("dd", "coarse without impedance", "            self.A0 = fem.a_xi(Kc, Mc, k, xi_prec, fem.assemble_B(cm) if self.imp else None)", "            self.A0 = fem.a_xi(Kc, Mc, k, xi_prec, None)"),
 ("dd", "box faces of the cube only", "        faces = boundary_faces(tets, mesh.n, tuple(lo), tuple(hi))", "        faces = boundary_faces(tets, mesh.n)"),
]

PINS = ["tests/test_oracle_mesh.py", "tests/test_oracle_fem.py", "tests/test_oracle_dd.py", "tests/test_oracle_gmres.py",
        "tests/test_oracle_imp.py", "tests/test_oracle_inexact.py", "tests/test_golden.py", "tests/test_zzz_full_size.py"]


def run_one(i, workdir):
    mod, label, old, new = MUTANTS[i]
    d = os.path.join(workdir, f"m{i:02d}")
    if os.path.exists(d):
        shutil.rmtree(d)
    os.makedirs(d)
    for sub in ("oracle", "tests", "inputs"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=shutil.ignore_patterns("__pycache__"))
    path = os.path.join(d, "oracle", mod + ".py")
    text = open(path).read()
    if text.count(old) != 1:
        return i, mod, label, None, "original text not found once: the oracle changed, update the mutant"
    with open(path, "w") as f:
        f.write(text.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                       cwd=d, env=env, capture_output=True, text=True, timeout=1800)
    failed = [line for line in r.stdout.splitlines() if line.startswith(("FAILED", "ERROR"))]
    return i, mod, label, r.returncode != 0, failed[0] if failed else ""


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=8)
    ap.add_argument("--only", default="", help="comma-separated mutant indices")
    ap.add_argument("--workdir", default=None)
    args = ap.parse_args()
    sel = [int(x) for x in args.only.split(",")] if args.only else list(range(len(MUTANTS)))
    workdir = args.workdir or tempfile.mkdtemp(prefix="oracle-mutants-")
    survivors = 0
    with ThreadPoolExecutor(args.jobs) as ex:
        for i, mod, label, killed, detail in ex.map(lambda j: run_one(j, workdir), sel):
            state = "KILLED" if killed else ("STALE" if killed is None else "SURVIVED")
            survivors += killed is not True
            print(f"m{i:02d} {mod:8s} {label:28s} {state:8s} {detail}", flush=True)
    if not args.workdir:
        shutil.rmtree(workdir, ignore_errors=True)
    print(f"{len(sel) - survivors} of {len(sel)} mutants killed")
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main())

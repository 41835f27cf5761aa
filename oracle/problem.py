"""build / factor / solve on the CPU, mirroring the library's three calls.

Oracle (test infrastructure only). Composes mesh, fem, dd and gmres; see their
docstrings for the passages of the paper each step follows.
"""
import numpy as np

from .mesh import KuhnMesh
from . import fem, dd, gmres as _gmres


class Problem:
    """curl curl E - (k^2 + i xi_prob) E = F, PEC, preconditioned by AS built from
    A_{xi_prec} (Sec. 6.2: B^{-1}_{xi_prec} preconditions A_{xi_prob})."""

    def __init__(self, n, k, xi_prob, xi_prec, core, overlap, coarse_m=0, kind="as", inner_coarse=None, bc="pec"):
        """inner_coarse: None (direct coarse solve) or a dict with core, overlap, tol, max_it,
        kind of the inner GMRES coarse solve (Sec. 6.4); the outer GMRES is then flexible.
        bc: "pec" (Eq. 1.4) or "imp" (Eq. imp; local problems with impedance conditions)."""
        self.kind = kind  # "as" (Eq. 3.4), "ras" (Eq. RAS2), "hras" (Eq. HRAS), "adef1" (Eq. ADEF1ras)
        self.mesh = KuhnMesh(n, bc)
        self.k, self.xi_prob, self.xi_prec = k, xi_prob, xi_prec
        self.K, self.M = fem.assemble_KM(self.mesh)
        self.B = fem.assemble_B(self.mesh) if bc == "imp" else None
        self.A = fem.a_xi(self.K, self.M, k, xi_prob, self.B)
        self.A_prec = fem.a_xi(self.K, self.M, k, xi_prec, self.B)
        self.dd = dd.Schwarz(self.mesh, self.A_prec, core, overlap, coarse_m, k, xi_prec)
        self.flexible = inner_coarse is not None
        if inner_coarse is not None:
            self.dd.set_inner_coarse(**inner_coarse)

    @property
    def n_dof(self):
        return self.mesh.n_dof

    def factor(self, subset=None):
        self.dd.factor(subset)

    def load_vector(self, centres, pol, width, q=3):
        """f for bump parameters centres [R, B, 3], pol [R, B, 3]; returns [n, R]."""
        return fem.load_vector(self.mesh, fem.bump_field(centres, pol, width), q)

    def solve(self, rhs, tol=1e-6, restart=0, max_it=200, history=None, weighted=False):
        """rhs [n] or [n, R]; each column solved independently. weighted: GMRES in the
        D_k = K + k^2 M inner product (Sec. 5.2)."""
        Dk = (self.K + self.k ** 2 * self.M).tocsr() if weighted else None
        weight = (lambda v: Dk @ v) if weighted else None
        rhs = np.asarray(rhs, dtype=np.complex128)
        single = rhs.ndim == 1
        B = rhs[:, None] if single else rhs
        xs, stats = [], []
        for r in range(B.shape[1]):
            hist = [] if history is not None else None
            x, its, rel, ok = _gmres.gmres(lambda v: self.A @ v, lambda v: self.dd.apply(v, kind=self.kind), B[:, r],
                                           tol, restart, max_it, history=hist, weight=weight, flexible=self.flexible)
            if history is not None:
                history.append(hist)
            xs.append(x)
            stats.append((its, rel, ok))
        X = np.stack(xs, axis=1)
        return (X[:, 0] if single else X), stats

"""Handle-owning convenience wrapper over the C ABI (build -> factor -> solve)."""
from . import _lib as L


class Problem:
    """One assembled operator A_{xi_prob} with its additive Schwarz preconditioner built
    from A_{xi_prec} (Eq. 3.4); see include/mxas.h for the meaning of every argument."""

    def __init__(self, n_cells, k, xi_prob, xi_prec, core_cells=5, overlap_cells=1, coarse_cells=0,
                 precision=L.MX_MIXED, stream=None, dense_local=False, bc=L.MX_BC_PEC):
        self.n_cells = n_cells
        self.h = L.mx_build_problem(n_cells, k, xi_prob, xi_prec, core_cells, overlap_cells, coarse_cells,
                                    precision, bc)
        if stream is not None:
            L.mx_set_stream(self.h, stream)
        if dense_local:
            L.mx_set_dense_local(self.h, True)
        self.factored = False

    @property
    def n_dof(self):
        return L.mx_num_dofs(self.h)

    def info(self):
        return L.mx_info(self.h)

    def timings(self):
        return L.mx_timings(self.h)

    def set_xi_prob(self, xi):
        L.mx_set_xi_prob(self.h, xi)

    def set_preconditioner(self, kind):
        L.mx_set_preconditioner(self.h, kind)

    def set_weighted_gmres(self, weighted=True):
        L.mx_set_weighted_gmres(self.h, weighted)

    def set_tuning(self, key, value):
        L.mx_set_tuning(self.h, key, value)

    def set_coarse_solver(self, kind, core_cells=1, overlap_cells=1, tol=0.1, max_it=100, prec_kind=L.MX_PREC_RAS):
        L.mx_set_coarse_solver(self.h, kind, core_cells, overlap_cells, tol, max_it, prec_kind)

    def factor(self):
        L.mx_factor(self.h)
        self.factored = True

    def load_vector(self, centres, pol, width, out=None):
        return L.mx_load_vector(self.h, centres, pol, width, out)

    def solve(self, rhs, tol=1e-6, restart=0, max_it=200, x=None):
        return L.mx_solve(self.h, rhs, tol, restart, max_it, x)

    def spmv(self, x, y=None):
        return L.mx_spmv(self.h, x, y)

    def spmv_mixed(self, x, y=None):
        return L.mx_spmv_mixed(self.h, x, y)

    def precond(self, v, z=None, levels=3):
        return L.mx_precond(self.h, v, z, levels)

    def close(self):
        if self.h:
            L.mx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

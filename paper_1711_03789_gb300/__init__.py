"""GB300 (sm_103a) additive-Schwarz preconditioned GMRES for the lowest-order Nedelec
discretisation of curl curl E - (k^2 + i xi) E = F on the unit cube with PEC boundary
conditions (Bonazzoli, Dolean, Graham, Spence, Tournier, arXiv:1711.03789).

This package is a thin ctypes binding of the C ABI declared in include/mxas.h: every
function has the name of the C entry point and only marshals arguments; all work runs in
the CUDA kernels of libmxas.so. Importing fails loudly if the library has not been built
(python -c "import __graft_entry__ as g; g.build()").

Vectors are complex128 arrays of shape [nrhs, n_dof] (one right-hand side per row), as
numpy arrays (host) or torch tensors (host or CUDA).
"""
from ._lib import (  # noqa: F401
    MX_OK, MX_EINVAL, MX_ENOMEM, MX_ENOTFACTORED, MX_ESINGULAR, MX_ENOCONV, MX_ETIMEOUT, MX_ECUDA,
    MX_PLAIN_FP64, MX_MIXED, MxError, lib, lib_path,
    mx_version, mx_last_error, mx_build_problem, mx_set_xi_prob, mx_set_stream, mx_set_dense_local,
    mx_factor, mx_load_vector, mx_solve, mx_num_dofs, mx_info, mx_timings, mx_destroy,
    mx_get_mesh, mx_get_subdomains, mx_get_csr, mx_get_coarse_restriction, mx_spmv, mx_spmv_mixed, mx_precond,
    mx_get_local, mx_set_allocator, use_torch_allocator,
    mx_launch_count, mx_profile, mx_profile_read, mx_profile_name, mx_dots, mx_dots_noalloc,
    mx_set_preconditioner, mx_set_weighted_gmres, MX_PREC_AS, MX_PREC_RAS, MX_PREC_HRAS, MX_PREC_ADEF1,
    mx_set_coarse_solver, MX_COARSE_DIRECT, MX_COARSE_GMRES, mx_get_boundary_mass, MX_BC_PEC, MX_BC_IMPEDANCE,
    mx_set_growth_limit, mx_test_bounded_wait,
    mx_set_tuning, MX_TUNE_LOCAL_RHS_GROUP, MX_TUNE_LU_TENSOR, MX_TUNE_COARSE_BLOCKS, MX_TUNE_LOCAL_TENSOR, MX_TUNE_COARSE_INVERSE,
    MX_TUNE_LU_GRID, MX_TUNE_DOTS,
    mx_server_create, mx_server_submit, mx_server_poll, mx_server_stats, mx_server_destroy, MX_PENDING,
)
from .problem import Problem  # noqa: F401

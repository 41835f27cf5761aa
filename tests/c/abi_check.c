/* C99 client of include/mxas.h, built and run by tests/test_abi.py without a GPU.
 * It checks that the header compiles as strict C and links against the library, then
 * exercises the argument checks that return before any device work, and prints the size
 * and field offsets of every struct of the ABI so the test can compare them with the
 * ctypes mirrors of the Python binding. Exit status 0 = every check held. */
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "mxas.h"

static int failures = 0;

static void expect(int cond, const char* what) {
  if (!cond) {
    fprintf(stderr, "FAILED: %s\n", what);
    ++failures;
  }
}

#define SIZE(T) printf("size %s %zu\n", #T, sizeof(T))
#define OFF(T, f) printf("offset %s.%s %zu\n", #T, #f, offsetof(T, f))

int main(void) {
  const char* v = mx_version();
  expect(v != NULL && strncmp(v, "mxas", 4) == 0, "mx_version starts with mxas");

  mx_mesh_desc mesh = {0, MX_BC_PEC};
  mx_dd_desc dd = {5, 1};
  mx_coarse_desc coarse = {0};
  mx_handle h = NULL;
  expect(mx_build_problem(&mesh, 1.0, 0.0, 1.0, &dd, &coarse, MX_MIXED, &h) == MX_EINVAL, "n_cells = 0 rejected");
  expect(h == NULL, "no handle on error");
  expect(mx_last_error() != NULL && mx_last_error()[0] != '\0', "error message set");
  mesh.n_cells = 10;
  expect(mx_build_problem(&mesh, -1.0, 0.0, 1.0, &dd, &coarse, MX_MIXED, &h) == MX_EINVAL, "k < 0 rejected");
  expect(mx_build_problem(&mesh, 1.0, 0.0, 1.0, &dd, &coarse, MX_MIXED, NULL) == MX_EINVAL, "null out rejected");
  expect(mx_build_problem(NULL, 1.0, 0.0, 1.0, &dd, &coarse, MX_MIXED, &h) == MX_EINVAL, "null mesh rejected");
  coarse.n_cells = 3; /* does not divide 10 */
  expect(mx_build_problem(&mesh, 1.0, 0.0, 1.0, &dd, &coarse, MX_MIXED, &h) == MX_EINVAL, "coarse must divide");

  /* null handles: errors, not crashes */
  expect(mx_num_dofs(NULL) == 0, "mx_num_dofs(NULL) = 0");
  mx_problem_info info;
  expect(mx_info(NULL, &info) == MX_EINVAL, "mx_info(NULL)");
  expect(mx_factor(NULL) == MX_EINVAL, "mx_factor(NULL)");
  expect(mx_spmv_mixed(NULL, NULL, NULL, 1) == MX_EINVAL, "mx_spmv_mixed(NULL)");
  expect(mx_set_tuning(NULL, MX_TUNE_LOCAL_TENSOR, 1) == MX_EINVAL, "mx_set_tuning(NULL)");
  expect(mx_set_preconditioner(NULL, MX_PREC_RAS) == MX_EINVAL, "mx_set_preconditioner(NULL)");
  expect(mx_set_growth_limit(NULL, 10.0) == MX_EINVAL, "mx_set_growth_limit(NULL)");
  expect(mx_test_bounded_wait(NULL, 16, 1) == MX_EINVAL, "mx_test_bounded_wait(NULL)");
  mx_destroy(NULL);

  mx_server srv = NULL;
  expect(mx_server_create(0, 1, &srv) == MX_EINVAL, "server budget 0 rejected");
  expect(mx_server_create(1 << 20, 0, &srv) == MX_EINVAL, "server workers 0 rejected");
  expect(srv == NULL, "no server on error");
  mx_server_info si;
  expect(mx_server_stats(NULL, &si) == MX_EINVAL, "mx_server_stats(NULL)");
  mx_server_destroy(NULL);

  expect(mx_profile_name(-1) != NULL && mx_profile_name(-1)[0] == '\0', "unknown kernel id has an empty name");
  expect(mx_profile_name(0) != NULL && mx_profile_name(0)[0] != '\0', "kernel id 0 has a name");

  SIZE(mx_mesh_desc);
  OFF(mx_mesh_desc, n_cells);
  OFF(mx_mesh_desc, boundary);
  SIZE(mx_dd_desc);
  OFF(mx_dd_desc, core_cells);
  OFF(mx_dd_desc, overlap_cells);
  SIZE(mx_coarse_desc);
  OFF(mx_coarse_desc, n_cells);
  SIZE(mx_problem_info);
  OFF(mx_problem_info, n_dof);
  OFF(mx_problem_info, nnz);
  OFF(mx_problem_info, n_sub);
  OFF(mx_problem_info, max_local);
  OFF(mx_problem_info, sum_local);
  OFF(mx_problem_info, n_coarse);
  OFF(mx_problem_info, nnz_r0);
  OFF(mx_problem_info, factor_bytes);
  OFF(mx_problem_info, coarse_band);
  OFF(mx_problem_info, precision);
  OFF(mx_problem_info, growth_subdomain);
  OFF(mx_problem_info, max_growth);
  SIZE(mx_rhs_stats);
  OFF(mx_rhs_stats, iterations);
  OFF(mx_rhs_stats, converged);
  OFF(mx_rhs_stats, rel_residual);
  OFF(mx_rhs_stats, rel_estimate);
  SIZE(mx_timing);
  OFF(mx_timing, build_ms);
  OFF(mx_timing, factor_ms);
  OFF(mx_timing, solve_ms);
  OFF(mx_timing, solve_launches);
  OFF(mx_timing, restarts);
  OFF(mx_timing, max_iterations);
  OFF(mx_timing, coarse_inner_iterations);
  OFF(mx_timing, coarse_inner_solves);
  SIZE(mx_request);
  OFF(mx_request, n_cells);
  OFF(mx_request, k);
  OFF(mx_request, xi_prob);
  OFF(mx_request, xi_prec);
  OFF(mx_request, core_cells);
  OFF(mx_request, overlap_cells);
  OFF(mx_request, coarse_cells);
  OFF(mx_request, precision);
  OFF(mx_request, nrhs);
  OFF(mx_request, nbumps);
  OFF(mx_request, centres);
  OFF(mx_request, pol);
  OFF(mx_request, width);
  OFF(mx_request, tol);
  OFF(mx_request, restart);
  OFF(mx_request, max_it);
  OFF(mx_request, boundary);
  OFF(mx_request, prec_kind);
  SIZE(mx_request_timing);
  OFF(mx_request_timing, latency_ms);
  OFF(mx_request_timing, queue_ms);
  OFF(mx_request_timing, n_dof);
  SIZE(mx_server_info);
  OFF(mx_server_info, batches);
  OFF(mx_server_info, factorisations);
  OFF(mx_server_info, evictions);
  OFF(mx_server_info, completed);
  OFF(mx_server_info, cached_bytes);
  OFF(mx_server_info, cached_operators);
  OFF(mx_server_info, pending);
  OFF(mx_server_info, waiting_for_memory);
  OFF(mx_server_info, joined);

  printf("failures %d\n", failures);
  return failures == 0 ? 0 : 1;
}

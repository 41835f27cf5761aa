// C ABI of the library (declared in include/mxas.h). Every entry point catches all
// exceptions, records a message for mx_last_error() and returns an MX_E* code.
#include <cstring>
#include <memory>

#include "problem.cuh"

namespace mx {
const char* last_error();
void set_allocator(alloc_fn a, free_fn f, void* ctx);
void prof_reset(bool on);
void prof_read(double* ms, int64_t* launches, double* bytes, double* flops);
int64_t launch_count();

Problem::~Problem() {
  free_workspace(*this);
  delete coarse_inner;
}

// ---- layout helpers -----------------------------------------------------------------
// user layout [nrhs][n] <-> solver layout [n][nrhs]
__global__ void k_to_internal(int64_t n, int nrhs, int r0, int nr, const double2* user, double2* in) {
  const int64_t work = n * nr;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nr);
    const int64_t i = t / nr;
    in[t] = user[(int64_t)(r0 + r) * n + i];
  }
}
__global__ void k_to_user(int64_t n, int nrhs, int r0, int nr, const double2* in, double2* user) {
  const int64_t work = n * nr;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nr);
    const int64_t i = t / nr;
    user[(int64_t)(r0 + r) * n + i] = in[t];
  }
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller buffer of `bytes`: the pointer itself if it is device memory,
// else a device copy (in) / a device staging buffer (out).
struct DevView {
  const void* user;
  bool device;
  DevBuf<unsigned char> tmp;
  void* p;
  DevView(const void* u, size_t bytes, bool copy_in, cudaStream_t s) : user(u) {
    device = is_device_ptr(u);
    if (device) {
      p = const_cast<void*>(u);
    } else {
      tmp.alloc(bytes);
      p = tmp.p;
      if (copy_in) MX_CUDA(cudaMemcpyAsync(p, u, bytes, cudaMemcpyHostToDevice, s));
    }
  }
  void copy_out(size_t bytes, cudaStream_t s) {
    if (!device) MX_CUDA(cudaMemcpyAsync(const_cast<void*>(user), p, bytes, cudaMemcpyDeviceToHost, s));
  }
};

struct EventTimer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit EventTimer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  double stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~EventTimer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

template <typename F>
static int guard(F&& f) {
  try {
    f();
    set_last_error("");
    return MX_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MX_ECUDA;
  } catch (...) {
    set_last_error("unknown error");
    return MX_ECUDA;
  }
}

// Pivot growth of the no-pivot local LU (Sec. 3.3 and Lemma 2.2 keep the pivots away from
// zero, not the growth bounded): for every subdomain max|U_ij| / max|A^l_ij| from the maxima
// the extraction and the factorisation kernels recorded; the largest is kept for mx_info, and
// a value above the limit returns MX_ESINGULAR (the factors would carry relative errors of
// the unit roundoff times the growth).
double growth_limit_of(const Problem& P) {
  return P.growth_limit > 0 ? P.growth_limit : (P.precision == MX_MIXED ? 1e6 : 1e12);
}

static void check_growth(Problem& P) {
  P.max_growth = 0;
  P.growth_worst = -1;
  if (!P.n_sub || P.amax.n != (size_t)P.n_sub || P.umax.n != (size_t)P.n_sub) return;
  std::vector<uint32_t> a(P.n_sub), u(P.n_sub);
  MX_CUDA(cudaMemcpyAsync(a.data(), P.amax.p, 4 * P.n_sub, cudaMemcpyDeviceToHost, P.stream));
  MX_CUDA(cudaMemcpyAsync(u.data(), P.umax.p, 4 * P.n_sub, cudaMemcpyDeviceToHost, P.stream));
  MX_CUDA(cudaStreamSynchronize(P.stream));
  for (int l = 0; l < P.n_sub; ++l) {
    float fa, fu;
    std::memcpy(&fa, &a[l], 4);
    std::memcpy(&fu, &u[l], 4);
    const double g = fa > 0 ? (double)fu / fa : (fu > 0 ? INFINITY : 0.0);
    if (!(g <= P.max_growth)) {  // also takes a NaN
      P.max_growth = g;
      P.growth_worst = l;
    }
  }
  const double lim = growth_limit_of(P);
  MX_REQUIRE(P.max_growth <= lim, MX_ESINGULAR,
             "pivot growth max|U| / max|A^l| = " + std::to_string(P.max_growth) + " in subdomain " +
                 std::to_string(P.growth_worst) + " exceeds the limit " + std::to_string(lim));
}

static void check_status(Problem& P) {
  int32_t st[4] = {0, 0, 0, 0};
  MX_CUDA(cudaMemcpyAsync(st, P.status.p, 16, cudaMemcpyDeviceToHost, P.stream));
  MX_CUDA(cudaStreamSynchronize(P.stream));
  MX_REQUIRE(st[0] == 0, MX_ESINGULAR, std::to_string(st[0]) + " zero or non-finite local pivots");
  MX_REQUIRE(st[1] == 0, MX_ESINGULAR, std::to_string(st[1]) + " zero or non-finite coarse pivots");
  MX_REQUIRE(st[2] == 0, MX_ETIMEOUT, std::to_string(st[2]) + " tensor-core waits ran out in the factorisation");
  check_growth(P);
}

void transpose_to_internal(const double2* user, double2* in, int64_t n, int nrhs, cudaStream_t s) {
  MX_LAUNCH(k_to_internal<<<grid_for(n * nrhs, 256), 256, 0, s>>>(n, nrhs, 0, nrhs, user, in));
  MX_CHECK_LAUNCH();
}

void transpose_to_user(const double2* in, double2* user, int64_t n, int nrhs, cudaStream_t s) {
  MX_LAUNCH(k_to_user<<<grid_for(n * nrhs, 256), 256, 0, s>>>(n, nrhs, 0, nrhs, in, user));
  MX_CHECK_LAUNCH();
}

Problem* create_problem(int n, double k, double xi_prob, double xi_prec, int core, int overlap, int cm, int precision,
                        cudaStream_t stream, int bc) {
  MX_REQUIRE(bc == MX_BC_PEC || bc == MX_BC_IMPEDANCE, MX_EINVAL, "unknown boundary condition");
  const bool imp = bc == MX_BC_IMPEDANCE;
  MX_REQUIRE(n >= 1 && n <= 256, MX_EINVAL, "n_cells must be in 1..256");
  MX_REQUIRE(core >= 1, MX_EINVAL, "core_cells must be >= 1");
  MX_REQUIRE(overlap >= 0 && overlap <= 6 * core, MX_EINVAL, "overlap_cells must be in 0..6*core_cells");
  MX_REQUIRE(k > 0 && std::isfinite(k), MX_EINVAL, "k must be > 0");
  MX_REQUIRE((imp || xi_prec != 0) && std::isfinite(xi_prec) && std::isfinite(xi_prob), MX_EINVAL,
             "xi_prec must be finite, and nonzero with PEC");
  MX_REQUIRE(precision == MX_MIXED || precision == MX_PLAIN_FP64, MX_EINVAL, "unknown precision");
  MX_REQUIRE(cm >= 0 && (cm == 0 || n % cm == 0), MX_EINVAL, "coarse n_cells must divide the fine n_cells");
  auto P = new Problem();
  try {
    P->n = n;
    P->k = k;
    P->xi_prob = xi_prob;
    P->xi_prec = xi_prec;
    P->core = core;
    P->overlap = overlap;
    P->coarse_m = cm;
    P->precision = precision;
    P->bc = bc;
    P->stream = stream;
    P->status.alloc(4);
    MX_CUDA(cudaMemsetAsync(P->status.p, 0, 16, P->stream));
    EventTimer t(P->stream);
    build_mesh(P->fine, P->n, P->stream, imp);
    MX_REQUIRE(P->fine.n_dof > 0, MX_EINVAL, "mesh has no interior edge");
    assemble_KM(P->fine, P->A, P->stream, imp);
    build_subdomains(*P);
    if (cm) {
      build_mesh(P->coarse, cm, P->stream, imp);
      MX_REQUIRE(P->coarse.n_dof > 0, MX_EINVAL, "coarse mesh has no interior edge (use n_cells >= 2)");
      assemble_KM(P->coarse, P->Ac, P->stream, imp);
      build_coarse_restriction(*P);
      P->n_c = P->coarse.n_dof;
    }
    P->timing.build_ms = t.stop();
  } catch (...) {
    delete P;
    throw;
  }
  return P;
}

void factor_problem(Problem& P) {
  MX_CUDA(cudaMemsetAsync(P.status.p, 0, 16, P.stream));
  EventTimer t(P.stream);
  extract_minors(P);
  if (P.coarse_inner) {
    factor_local(P);
    P.coarse_inner->stream = P.stream;
    factor_problem(*P.coarse_inner);  // the inner coarse GMRES replaces the direct factors
  } else {
    // in sequence: running the coarse factorisation on a second stream during the local LU
    // shortens this phase by about a tenth but leaves no per-kernel device time to measure
    factor_local(P);
    factor_coarse(P);
    P.coarse_factored = P.coarse_m > 0;
  }
  P.timing.factor_ms = t.stop();
  try {
    check_status(P);
  } catch (...) {
    // a singular, over-grown or timed-out factorisation is not used: the handle needs a
    // successful mx_factor before the next solve
    P.factored = false;
    P.coarse_factored = false;
    throw;
  }
}

}  // namespace mx

using namespace mx;

extern "C" {

const char* mx_version(void) { return "mxas 0.1 (sm_103a)"; }

const char* mx_last_error(void) { return mx::last_error(); }

int mx_set_allocator(void* (*alloc)(size_t, void*), void (*release)(void*, void*), void* ctx) {
  return guard([&] { set_allocator(alloc, release, ctx); });
}

int mx_build_problem(const mx_mesh_desc* mesh, double k, double xi_prob, double xi_prec, const mx_dd_desc* dd,
                     const mx_coarse_desc* coarse, int precision, mx_handle* out) {
  return guard([&] {
    MX_REQUIRE(mesh && dd && out, MX_EINVAL, "null descriptor");
    Problem* P = create_problem(mesh->n_cells, k, xi_prob, xi_prec, dd->core_cells, dd->overlap_cells,
                                coarse ? coarse->n_cells : 0, precision, nullptr, mesh->boundary);
    *out = reinterpret_cast<mx_handle>(P);
  });
}

int mx_set_xi_prob(mx_handle h, double xi_prob) {
  return guard([&] {
    MX_REQUIRE(h && std::isfinite(xi_prob), MX_EINVAL, "bad handle or xi_prob");
    reinterpret_cast<Problem*>(h)->xi_prob = xi_prob;
  });
}

int mx_set_stream(mx_handle h, void* stream) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    auto& P = *reinterpret_cast<Problem*>(h);
    P.stream = reinterpret_cast<cudaStream_t>(stream);
    if (P.coarse_inner) P.coarse_inner->stream = P.stream;
  });
}

int mx_set_dense_local(mx_handle h, int dense) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    auto& P = *reinterpret_cast<Problem*>(h);
    P.dense_local = dense != 0;
    P.minors_ready = false;
    P.factored = false;
  });
}

int mx_set_growth_limit(mx_handle h, double limit) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    MX_REQUIRE(!std::isnan(limit), MX_EINVAL, "growth limit is NaN");
    reinterpret_cast<Problem*>(h)->growth_limit = limit > 0 ? limit : 0;
  });
}

int mx_test_bounded_wait(mx_handle h, int limit, int blocks) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    MX_REQUIRE(limit >= 1 && limit <= (1 << 20), MX_EINVAL, "limit must be in 1..2^20");
    MX_REQUIRE(blocks >= 1 && blocks <= 1024, MX_EINVAL, "blocks must be in 1..1024");
    auto& P = *reinterpret_cast<Problem*>(h);
    const int32_t timeouts = wait_probe(P, limit, blocks);
    MX_REQUIRE(timeouts == 0, MX_ETIMEOUT, std::to_string(timeouts) + " bounded waits ran out (probe)");
  });
}

int mx_set_tuning(mx_handle h, int key, int value) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    auto& P = *reinterpret_cast<Problem*>(h);
    if (key == MX_TUNE_LOCAL_RHS_GROUP) {
      MX_REQUIRE(value == 0 || (value >= 1 && value <= 16 && (value & (value - 1)) == 0), MX_EINVAL,
                 "local rhs group must be 0 or a power of two in 1..16");
      P.tune_local_group = value;
    } else if (key == MX_TUNE_COARSE_BLOCKS) {
      MX_REQUIRE(value >= 0 && value <= 4096, MX_EINVAL, "coarse blocks must be in 0..4096");
      P.tune_coarse_blocks = value;
    } else if (key == MX_TUNE_LU_TENSOR) {
      MX_REQUIRE(value >= 0 && value <= 4, MX_EINVAL, "LU tensor mode must be in 0..4");
      P.tune_lu_tc = value;
    } else if (key == MX_TUNE_LU_GRID) {
      MX_REQUIRE(value >= 0 && value <= 65536, MX_EINVAL, "LU grid must be in 0..65536");
      P.tune_lu_grid = value;
    } else if (key == MX_TUNE_COARSE_INVERSE) {
      MX_REQUIRE(value >= 0 && value <= 2, MX_EINVAL, "coarse inverse mode must be 0, 1 or 2");
      P.tune_coarse_inverse = value;
    } else if (key == MX_TUNE_DOTS) {
      MX_REQUIRE(value == 0 || value == 1, MX_EINVAL, "dots mode must be 0 or 1");
      P.tune_dots = value;
    } else if (key == MX_TUNE_LOCAL_TENSOR) {
      MX_REQUIRE(value == 0 || value == 1, MX_EINVAL, "local tensor mode must be 0 or 1");
      P.tune_local_tc = value;
    } else {
      throw Error(MX_EINVAL, "unknown tuning key " + std::to_string(key));
    }
  });
}

int mx_set_preconditioner(mx_handle h, int kind) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    MX_REQUIRE(kind >= MX_PREC_AS && kind <= MX_PREC_ADEF1, MX_EINVAL, "unknown preconditioner variant");
    auto& P = *reinterpret_cast<Problem*>(h);
    if (kind != MX_PREC_AS) {
      MX_REQUIRE(P.overlap >= 1, MX_EINVAL, "the restricted variants need an overlap of at least one cell");
      MX_REQUIRE(kind == MX_PREC_RAS || P.coarse_m > 0, MX_EINVAL, "HRAS and ADEF1 need a coarse level");
    }
    P.prec_kind = kind;
  });
}

int mx_set_coarse_solver(mx_handle h, int kind, const mx_dd_desc* dd, double tol, int max_it, int prec_kind) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    auto& P = *reinterpret_cast<Problem*>(h);
    MX_REQUIRE(kind == MX_COARSE_DIRECT || kind == MX_COARSE_GMRES, MX_EINVAL, "unknown coarse solver");
    MX_REQUIRE(P.coarse_m > 0, MX_EINVAL, "the handle has no coarse level");
    if (kind == MX_COARSE_DIRECT) {
      if (P.factored && !P.coarse_factored) {
        MX_CUDA(cudaMemsetAsync(P.status.p, 0, 16, P.stream));
        factor_coarse(P);
        check_status(P);
        P.coarse_factored = true;
      }
      delete P.coarse_inner;
      P.coarse_inner = nullptr;
      return;
    }
    MX_REQUIRE(dd, MX_EINVAL, "null subdomain description");
    MX_REQUIRE(tol > 0 && tol < 1, MX_EINVAL, "inner tolerance must be in (0, 1)");
    MX_REQUIRE(max_it >= 1 && max_it <= 1000, MX_EINVAL, "inner max_it must be in 1..1000");
    MX_REQUIRE(prec_kind == MX_PREC_AS || prec_kind == MX_PREC_RAS, MX_EINVAL,
               "the inner preconditioner is one-level AS or RAS");
    MX_REQUIRE(prec_kind == MX_PREC_AS || dd->overlap_cells >= 1, MX_EINVAL,
               "RAS needs an overlap of at least one cell");
    std::unique_ptr<Problem> Q(create_problem(P.coarse_m, P.k, P.xi_prec, P.xi_prec, dd->core_cells,
                                              dd->overlap_cells, 0, P.precision, P.stream, P.bc));
    Q->prec_kind = prec_kind;
    if (P.factored) factor_problem(*Q);
    delete P.coarse_inner;
    P.coarse_inner = Q.release();
    P.c_tol = tol;
    P.c_max_it = max_it;
  });
}

int mx_set_weighted_gmres(mx_handle h, int weighted) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    MX_REQUIRE(weighted == 0 || weighted == 1, MX_EINVAL, "weighted must be 0 or 1");
    reinterpret_cast<Problem*>(h)->weighted = weighted != 0;
  });
}

int mx_factor(mx_handle h) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    factor_problem(*reinterpret_cast<Problem*>(h));
  });
}

int mx_load_vector(mx_handle h, int nrhs, int nbumps, const double* centres, const double* pol, double width,
                   void* f) {
  return guard([&] {
    MX_REQUIRE(h && centres && pol && f, MX_EINVAL, "null argument");
    MX_REQUIRE(nrhs >= 1 && nbumps >= 1 && width > 0, MX_EINVAL, "bad sizes");
    auto& P = *reinterpret_cast<Problem*>(h);
    const size_t bytes = (size_t)nrhs * P.fine.n_dof * sizeof(double2);
    DevView out(f, bytes, false, P.stream);
    load_vector(P, nrhs, nbumps, centres, pol, width, reinterpret_cast<double2*>(out.p));
    out.copy_out(bytes, P.stream);
    MX_CUDA(cudaStreamSynchronize(P.stream));
  });
}

int mx_solve(mx_handle h, const void* rhs, int nrhs, double tol, int restart, int max_it, void* x,
             mx_rhs_stats* stats) {
  int rc = MX_OK;
  int g = guard([&] {
    MX_REQUIRE(h && rhs && x, MX_EINVAL, "null argument");
    MX_REQUIRE(nrhs >= 1 && tol > 0 && restart >= 0 && max_it >= 1, MX_EINVAL, "bad solve arguments");
    auto& P = *reinterpret_cast<Problem*>(h);
    MX_REQUIRE(P.factored, MX_ENOTFACTORED, "mx_solve before mx_factor");
    const int64_t n = P.fine.n_dof;
    const size_t bytes = (size_t)nrhs * n * sizeof(double2);
    EventTimer t(P.stream);
    P.timing.coarse_inner_iterations = 0;
    P.timing.coarse_inner_solves = 0;
    DevView in(rhs, bytes, true, P.stream);
    DevView out(x, bytes, false, P.stream);
    const int batch = 32;
    DevBuf<double2> bi((size_t)n * std::min(nrhs, batch)), xi((size_t)n * std::min(nrhs, batch));
    int64_t launches = 0;
    int maxit = 0, restarts = 0;
    for (int r0 = 0; r0 < nrhs; r0 += batch) {
      const int nr = std::min(batch, nrhs - r0);
      MX_LAUNCH(k_to_internal<<<grid_for(n * nr, 256), 256, 0, P.stream>>>(n, nrhs, r0, nr, (const double2*)in.p, bi.p));
      MX_CHECK_LAUNCH();
      const int c = gmres_solve(P, bi.p, xi.p, nr, tol, restart, max_it, stats ? stats + r0 : nullptr);
      if (c != MX_OK) rc = c;
      MX_LAUNCH(k_to_user<<<grid_for(n * nr, 256), 256, 0, P.stream>>>(n, nrhs, r0, nr, xi.p, (double2*)out.p));
      MX_CHECK_LAUNCH();
      launches += P.timing.solve_launches + 2;
      maxit = std::max(maxit, P.timing.max_iterations);
      restarts += P.timing.restarts;
    }
    out.copy_out(bytes, P.stream);
    P.timing.solve_ms = t.stop();
    P.timing.solve_launches = launches;
    P.timing.max_iterations = maxit;
    P.timing.restarts = restarts;
  });
  if (g != MX_OK) return g;
  if (rc != MX_OK) set_last_error("GMRES did not reach the tolerance for every right-hand side");
  return rc;
}

int64_t mx_num_dofs(mx_handle h) { return h ? reinterpret_cast<Problem*>(h)->fine.n_dof : 0; }

int mx_info(mx_handle h, mx_problem_info* out) {
  return guard([&] {
    MX_REQUIRE(h && out, MX_EINVAL, "null argument");
    auto& P = *reinterpret_cast<Problem*>(h);
    std::memset(out, 0, sizeof(*out));
    out->n_dof = P.fine.n_dof;
    out->nnz = P.A.nnz;
    out->n_sub = P.n_sub;
    out->max_local = P.max_local;
    out->sum_local = P.sum_local;
    out->n_coarse = P.coarse_m ? P.coarse.n_dof : 0;
    out->nnz_r0 = P.R0.nnz;
    out->factor_bytes = (int64_t)P.factors.bytes() + (int64_t)P.dinv.bytes() + (int64_t)P.panels.bytes() +
                        (int64_t)P.A0.bytes() + (int64_t)P.A0f.bytes() + (int64_t)P.A0inv.bytes();
    if (const Problem* Q = P.coarse_inner)
      out->factor_bytes += (int64_t)Q->factors.bytes() + (int64_t)Q->dinv.bytes() + (int64_t)Q->panels.bytes();
    out->coarse_band = P.coarse_band;
    out->precision = P.precision;
    out->growth_subdomain = P.growth_worst;
    out->max_growth = P.max_growth;
  });
}

int mx_timings(mx_handle h, mx_timing* out) {
  return guard([&] {
    MX_REQUIRE(h && out, MX_EINVAL, "null argument");
    auto& P = *reinterpret_cast<Problem*>(h);
    out->build_ms = P.timing.build_ms;
    out->factor_ms = P.timing.factor_ms;
    out->solve_ms = P.timing.solve_ms;
    out->solve_launches = P.timing.solve_launches;
    out->restarts = P.timing.restarts;
    out->max_iterations = P.timing.max_iterations;
    out->coarse_inner_iterations = P.timing.coarse_inner_iterations;
    out->coarse_inner_solves = P.timing.coarse_inner_solves;
  });
}

void mx_destroy(mx_handle h) {
  if (!h) return;
  auto* P = reinterpret_cast<Problem*>(h);
  cudaStreamSynchronize(P->stream);
  delete P;
}

int mx_get_mesh(mx_handle h, int32_t* dof_key, int32_t* tet2dof) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    auto& P = *reinterpret_cast<Problem*>(h);
    if (dof_key) MX_CUDA(cudaMemcpy(dof_key, P.fine.dof_key.p, P.fine.n_dof * 4, cudaMemcpyDeviceToHost));
    if (tet2dof) MX_CUDA(cudaMemcpy(tet2dof, P.fine.tet2dof.p, P.fine.tet2dof.bytes(), cudaMemcpyDeviceToHost));
  });
}

int mx_get_subdomains(mx_handle h, int64_t* offsets, int32_t* lists, int32_t* inv_ptr, int32_t* inv_pos) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    auto& P = *reinterpret_cast<Problem*>(h);
    if (offsets) std::memcpy(offsets, P.h_offsets.data(), (P.n_sub + 1) * 8);
    if (lists) MX_CUDA(cudaMemcpy(lists, P.lists.p, P.sum_local * 4, cudaMemcpyDeviceToHost));
    if (inv_ptr) MX_CUDA(cudaMemcpy(inv_ptr, P.inv_ptr.p, (P.fine.n_dof + 1) * 4, cudaMemcpyDeviceToHost));
    if (inv_pos) MX_CUDA(cudaMemcpy(inv_pos, P.inv_pos.p, P.sum_local * 4, cudaMemcpyDeviceToHost));
  });
}

int mx_get_csr(mx_handle h, int which, int32_t* rowptr, int32_t* col, double* K, double* M) {
  return guard([&] {
    MX_REQUIRE(h && (which == 0 || which == 1), MX_EINVAL, "bad arguments");
    auto& P = *reinterpret_cast<Problem*>(h);
    CsrKM& A = which == 0 ? P.A : P.Ac;
    MX_REQUIRE(which == 0 || P.coarse_m, MX_EINVAL, "no coarse space");
    if (rowptr) MX_CUDA(cudaMemcpy(rowptr, A.rowptr.p, (A.rows + 1) * 4, cudaMemcpyDeviceToHost));
    if (col) MX_CUDA(cudaMemcpy(col, A.col.p, A.nnz * 4, cudaMemcpyDeviceToHost));
    if (K) MX_CUDA(cudaMemcpy(K, A.K.p, A.nnz * 8, cudaMemcpyDeviceToHost));
    if (M) MX_CUDA(cudaMemcpy(M, A.M.p, A.nnz * 8, cudaMemcpyDeviceToHost));
  });
}

int mx_get_boundary_mass(mx_handle h, int which, double* B) {
  return guard([&] {
    MX_REQUIRE(h && B && (which == 0 || which == 1), MX_EINVAL, "bad arguments");
    auto& P = *reinterpret_cast<Problem*>(h);
    MX_REQUIRE(which == 0 || P.coarse_m, MX_EINVAL, "no coarse space");
    CsrKM& A = which == 0 ? P.A : P.Ac;
    if (A.B.p) MX_CUDA(cudaMemcpy(B, A.B.p, A.nnz * 8, cudaMemcpyDeviceToHost));
    else std::memset(B, 0, A.nnz * 8);
  });
}

int mx_get_coarse_restriction(mx_handle h, int32_t* rowptr, int32_t* col, double* val) {
  return guard([&] {
    MX_REQUIRE(h, MX_EINVAL, "null handle");
    auto& P = *reinterpret_cast<Problem*>(h);
    MX_REQUIRE(P.coarse_m, MX_EINVAL, "no coarse space");
    if (rowptr) MX_CUDA(cudaMemcpy(rowptr, P.R0.rowptr.p, (P.R0.rows + 1) * 4, cudaMemcpyDeviceToHost));
    if (col) MX_CUDA(cudaMemcpy(col, P.R0.col.p, P.R0.nnz * 4, cudaMemcpyDeviceToHost));
    if (val) MX_CUDA(cudaMemcpy(val, P.R0.val.p, P.R0.nnz * 8, cudaMemcpyDeviceToHost));
  });
}

int mx_spmv(mx_handle h, const void* x, void* y, int nrhs) {
  return guard([&] {
    MX_REQUIRE(h && x && y && nrhs >= 1, MX_EINVAL, "bad arguments");
    auto& P = *reinterpret_cast<Problem*>(h);
    const int64_t n = P.fine.n_dof;
    const size_t bytes = (size_t)nrhs * n * sizeof(double2);
    DevView in(x, bytes, true, P.stream);
    DevView out(y, bytes, false, P.stream);
    DevBuf<double2> a((size_t)n * nrhs), b((size_t)n * nrhs);
    MX_LAUNCH(k_to_internal<<<grid_for(n * nrhs, 256), 256, 0, P.stream>>>(n, nrhs, 0, nrhs, (const double2*)in.p, a.p));
    spmv(P, P.xi_prob, a.p, 0, b.p, nrhs, P.stream);
    MX_LAUNCH(k_to_user<<<grid_for(n * nrhs, 256), 256, 0, P.stream>>>(n, nrhs, 0, nrhs, b.p, (double2*)out.p));
    MX_CHECK_LAUNCH();
    out.copy_out(bytes, P.stream);
    MX_CUDA(cudaStreamSynchronize(P.stream));
  });
}

int mx_spmv_mixed(mx_handle h, const void* x, void* y, int nrhs) {
  return guard([&] {
    MX_REQUIRE(h && x && y && nrhs >= 1, MX_EINVAL, "bad arguments");
    auto& P = *reinterpret_cast<Problem*>(h);
    const int64_t n = P.fine.n_dof, cnt = n * nrhs;
    const size_t bytes = (size_t)cnt * sizeof(double2);
    DevView in(x, bytes, true, P.stream);
    DevView out(y, bytes, false, P.stream);
    DevBuf<double2> a((size_t)cnt), b((size_t)cnt);
    DevBuf<float2> z((size_t)cnt);
    DevBuf<float4> w((size_t)cnt);
    MX_LAUNCH(k_to_internal<<<grid_for(cnt, 256), 256, 0, P.stream>>>(n, nrhs, 0, nrhs, (const double2*)in.p, a.p));
    MX_CHECK_LAUNCH();
    c128_to_c64(a.p, z.p, cnt, P.stream);
    spmv_df(P, z.p, w.p, nrhs, P.stream);
    df_to_c128(w.p, b.p, cnt, P.stream);
    MX_LAUNCH(k_to_user<<<grid_for(cnt, 256), 256, 0, P.stream>>>(n, nrhs, 0, nrhs, b.p, (double2*)out.p));
    MX_CHECK_LAUNCH();
    out.copy_out(bytes, P.stream);
    MX_CUDA(cudaStreamSynchronize(P.stream));
  });
}

int mx_precond(mx_handle h, const void* v, void* z, int nrhs, int levels) {
  return guard([&] {
    MX_REQUIRE(h && v && z && nrhs >= 1 && nrhs <= 32 && levels >= 1 && levels <= 3, MX_EINVAL, "bad arguments");
    auto& P = *reinterpret_cast<Problem*>(h);
    MX_REQUIRE(P.factored, MX_ENOTFACTORED, "mx_precond before mx_factor");
    const int64_t n = P.fine.n_dof;
    const size_t bytes = (size_t)nrhs * n * sizeof(double2);
    DevView in(v, bytes, true, P.stream);
    DevView out(z, bytes, false, P.stream);
    DevBuf<double2> a((size_t)n * nrhs), b((size_t)n * nrhs);
    MX_CUDA(cudaMemsetAsync(P.status.p + 2, 0, sizeof(int32_t), P.stream));  // timed-out waits, as in mx_solve
    MX_LAUNCH(k_to_internal<<<grid_for(n * nrhs, 256), 256, 0, P.stream>>>(n, nrhs, 0, nrhs, (const double2*)in.p, a.p));
    precond_apply(P, a.p, b.p, 0, nrhs, levels);
    MX_LAUNCH(k_to_user<<<grid_for(n * nrhs, 256), 256, 0, P.stream>>>(n, nrhs, 0, nrhs, b.p, (double2*)out.p));
    MX_CHECK_LAUNCH();
    out.copy_out(bytes, P.stream);
    int32_t timeouts = 0;
    MX_CUDA(cudaMemcpyAsync(&timeouts, P.status.p + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, P.stream));
    MX_CUDA(cudaStreamSynchronize(P.stream));
    MX_REQUIRE(timeouts == 0, MX_ETIMEOUT, std::to_string(timeouts) + " tensor-core waits ran out in the local solves");
  });
}

int mx_dots(const void* V, const void* w, int64_t n, int nrhs, int nvec, void* h, void* stream) {
  return guard([&] {
    MX_REQUIRE(V && w && h && n >= 1 && nrhs >= 1 && nrhs <= 32 && nvec >= 1, MX_EINVAL, "bad mx_dots arguments");
    MX_REQUIRE(is_device_ptr(V) && is_device_ptr(w), MX_EINVAL, "mx_dots: V and w must be device memory");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nblk = 2 * sm_count();
    DevBuf<double2> partials((size_t)nblk * nvec * nrhs), res((size_t)nvec * nrhs);
    DevBuf<int32_t> ones(nrhs);
    fill_i32(ones.p, nrhs, 1, s);
    batched_dots((const double2*)V, (const double2*)w, n, nrhs, nvec, res.p, partials.p, nblk, ones.p, s);
    MX_CUDA(cudaMemcpyAsync(h, res.p, res.bytes(), cudaMemcpyDefault, s));
    MX_CUDA(cudaStreamSynchronize(s));
  });
}

int mx_profile(int enable) {
  return guard([&] { prof_reset(enable != 0); });
}

int mx_profile_read(double* ms, int64_t* launches, double* bytes, double* flops) {
  int n = K_COUNT;
  int rc = guard([&] { prof_read(ms, launches, bytes, flops); });
  return rc == MX_OK ? n : rc;
}

const char* mx_profile_name(int id) { return kernel_name(id); }

int64_t mx_launch_count(void) { return launch_count(); }

int mx_get_local(mx_handle h, int l, double* out) {
  return guard([&] {
    MX_REQUIRE(h && out, MX_EINVAL, "null argument");
    auto& P = *reinterpret_cast<Problem*>(h);
    MX_REQUIRE(l >= 0 && l < P.n_sub, MX_EINVAL, "subdomain index out of range");
    if (!P.factored && !P.minors_ready) extract_minors(P);
    const int nl = P.h_nl[l], b = P.h_band[l], ld = P.h_ld[l];
    const bool mixed = P.precision == MX_MIXED;
    const size_t esz = mixed ? 8 : 16;
    std::vector<unsigned char> band((size_t)ld * nl * esz);
    MX_CUDA(cudaMemcpy(band.data(), P.factors.p + (size_t)P.h_mat_off[l] * esz, band.size(), cudaMemcpyDeviceToHost));
    std::memset(out, 0, (size_t)nl * nl * 16);
    for (int j = 0; j < nl; ++j)
      for (int i = std::max(0, j - b); i <= std::min(nl - 1, j + b); ++i) {
        const size_t src = (size_t)j * ld + (b + i - j);
        double re, im;
        if (mixed) {
          const float* f = reinterpret_cast<const float*>(band.data()) + 2 * src;
          re = f[0];
          im = f[1];
        } else {
          const double* d = reinterpret_cast<const double*>(band.data()) + 2 * src;
          re = d[0];
          im = d[1];
        }
        out[2 * ((size_t)j * nl + i)] = re;
        out[2 * ((size_t)j * nl + i) + 1] = im;
      }
  });
}

}  // extern "C"

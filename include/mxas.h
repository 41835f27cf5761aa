/*
 * mxas.h -- C ABI of the GB300 additive-Schwarz / GMRES solver for the lowest-order
 * Nedelec discretisation of  curl curl E - (k^2 + i xi) E = F  on the unit cube with
 * PEC boundary conditions (Bonazzoli, Dolean, Graham, Spence, Tournier,
 * arXiv:1711.03789).
 *
 * Conventions shared by every call
 *   - Complex numbers are interleaved (re, im) pairs: double2 ("c128") or float2
 *     ("c64"). A block of right-hand sides is stored right-hand side by right-hand
 *     side: element (i, r) of an n x nrhs block is at index r * n + i.
 *   - Pointers to vectors may be host or device memory; the library asks the CUDA
 *     runtime which (cudaPointerGetAttributes) and copies through the handle's stream.
 *     Host pointers are read before the call returns; results are in place when it
 *     returns (the call synchronises the handle's stream).
 *   - Ownership: the library owns the handle and every device buffer it allocates;
 *     the caller owns every pointer it passes and may free it when the call returns.
 *   - Errors: every int-returning call returns MX_OK (0) or a negative MX_E* code and
 *     never throws; mx_last_error() gives a message for the calling thread.
 *   - Threads: one handle must not be used by two threads at once; different handles
 *     are independent.
 */
#ifndef MXAS_H
#define MXAS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MX_API __attribute__((visibility("default")))
#else
#define MX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MX_OK 0
#define MX_EINVAL (-1)        /* bad argument or descriptor */
#define MX_ENOMEM (-2)        /* device allocation failed or over the memory budget */
#define MX_ENOTFACTORED (-3)  /* mx_solve / mx_precond before mx_factor */
#define MX_ESINGULAR (-4)     /* a zero or tiny pivot in a local or coarse LU */
#define MX_ENOCONV (-5)       /* GMRES reached max_it; x and stats are still filled */
#define MX_ETIMEOUT (-6)      /* a bounded device wait expired */
#define MX_ECUDA (-7)         /* a CUDA runtime error; see mx_last_error() */

/* Mesh: the unit cube split into n_cells^3 cubes, each cut into 6 Kuhn tetrahedra
 * (Sec. 2.2; uniform mesh and Kuhn split are this library's reading).
 * boundary: MX_BC_PEC (Eq. 1.4; the edges on the boundary carry no DOF) or
 * MX_BC_IMPEDANCE (Eq. imp: curl E x n - i sign(xi) k (n x E) x n = 0 with sign(0) = +1;
 * every edge is a DOF and A_xi = K - (k^2 + i xi) M - i sign(xi) k B, B the tangential
 * Whitney mass of the boundary triangles). With MX_BC_IMPEDANCE the local problems of the
 * preconditioner are those of ImpRAS (Sec. 6.3): the Maxwell problem on each closed
 * subdomain box with the impedance condition on the whole box boundary, on the DOFs of
 * all edges of the closed box; every preconditioner variant is built from them (ImpAS,
 * ImpRAS, ImpHRAS, ADEF1-ImpRAS), and the coarse problem is the impedance problem on the
 * coarse mesh. */
#define MX_BC_PEC 0
#define MX_BC_IMPEDANCE 1
typedef struct {
  int n_cells;
  int boundary;
} mx_mesh_desc;

/* Overlapping subdomains (Sec. 3.1, Sec. 6.1): boxes of core_cells^3 cells widened by
 * overlap_cells on each side, clipped to the cube. */
typedef struct { int core_cells; int overlap_cells; } mx_dd_desc;

/* Coarse space (Sec. 3.2): a Kuhn mesh of n_cells^3 cells; n_cells must divide the
 * fine n_cells (nested meshes). n_cells = 0 gives the one-level preconditioner. */
typedef struct { int n_cells; } mx_coarse_desc;

/* Precision of the preconditioner and of the Krylov process.
 *   MX_PLAIN_FP64: FP64 throughout (c128 local and coarse factors, FP64 Krylov kernels).
 *   MX_MIXED: c64 local factors (from a tcgen05 LU with three TF32 products per term; local
 *     solves on tcgen05 TF32 with the right-hand-side block as a TF32 hi + lo pair, or FP32
 *     CUDA cores); c64 coarse band LU and its explicit c64 inverse, applied on tcgen05 with
 *     three TF32 products per term; FP32 scatter; the load vector's quadrature in
 *     double-float arithmetic. The Krylov basis V, the products A z_j and both classical
 *     Gram-Schmidt passes use double-float arithmetic (pairs of FP32 values, about 48
 *     significant bits; the first pass forms its products from the c64 rounding of V).
 *     FP64 is kept for H, the Givens rotations, the least-squares solve, the solution x
 *     and the true residual b - A x at every restart and at the end, which the stopping
 *     test uses. GMRES is flexible (the stored z_j enter x), so the c64 preconditioner
 *     changes the iteration count, not the FP64 residual the solve stops at.
 *   The mixed form departs from an FP64 Arnoldi process and an FP64 coarse factorisation
 *   because FP64 runs at about 1/64 of the FP32 rate on GB300. */
typedef enum { MX_PLAIN_FP64 = 0, MX_MIXED = 1 } mx_precision;

typedef struct mx_problem* mx_handle;

typedef struct {
  int64_t n_dof;        /* DOFs of the fine mesh: PEC-interior edges, or all edges (impedance) */
  int64_t nnz;          /* nonzeros of A (CSR) */
  int32_t n_sub;        /* number of subdomains N */
  int32_t max_local;    /* largest subdomain size n_l */
  int64_t sum_local;    /* sum of n_l */
  int64_t n_coarse;     /* coarse DOFs (0 for one level) */
  int64_t nnz_r0;       /* nonzeros of R^0 */
  int64_t factor_bytes; /* device bytes held by local + coarse factors */
  int32_t coarse_band;  /* half-bandwidth of the coarse matrix */
  int32_t precision;
  int32_t growth_subdomain; /* subdomain with the largest pivot growth (-1 before mx_factor) */
  double max_growth;    /* largest max|U_ij| / max|A^l_ij| over the local LUs of the last mx_factor */
} mx_problem_info;

typedef struct {
  int32_t iterations;   /* GMRES iterations (Arnoldi steps) over all restarts */
  int32_t converged;    /* 1 when ||b - A x|| / ||b|| <= tol in FP64 */
  double rel_residual;  /* final true relative residual ||b - A x||_2 / ||b||_2 */
  double rel_estimate;  /* last least-squares residual estimate |g_{j+1}| / ||b|| */
} mx_rhs_stats;

typedef struct {
  double build_ms, factor_ms, solve_ms;   /* device time of the last calls */
  int64_t solve_launches;                 /* kernels launched by the last mx_solve */
  int32_t restarts;
  int32_t max_iterations;
  int64_t coarse_inner_iterations;        /* MX_COARSE_GMRES: inner iterations of the last mx_solve
                                             (for each coarse solve, the most any right-hand side took) */
  int64_t coarse_inner_solves;            /* MX_COARSE_GMRES: coarse solves of the last mx_solve */
} mx_timing;

/* Library version string. */
MX_API const char* mx_version(void);

/* Route every device allocation of the library through alloc/release (for instance a
 * framework's caching allocator); ctx is passed back unchanged. NULL restores cudaMalloc /
 * cudaFree. Must not be changed while a handle holds memory from the previous hooks. */
MX_API int mx_set_allocator(void* (*alloc)(size_t bytes, void* ctx), void (*release)(void* p, void* ctx),
                     void* ctx);

/* Store the local factors as full dense matrices (half-bandwidth n_l - 1) instead of the
 * band (both give the same factors: no-pivot LU creates no fill outside the band). Takes
 * effect at the next mx_factor. For comparison runs. */
MX_API int mx_set_dense_local(mx_handle h, int dense);

/* Tuning knobs (the Python binding's autotune module searches them per problem shape);
 * value 0 restores the default.
 *   MX_TUNE_LOCAL_RHS_GROUP: most right-hand sides one local-solve block handles
 *   (power of two, 1..16; default 16). Smaller groups run more blocks per subdomain. */
#define MX_TUNE_LOCAL_RHS_GROUP 1
/*   MX_TUNE_LU_TENSOR: the MX_MIXED local LU. 0 (default) or 2 = one persistent launch, one
 *   CTA per subdomain running all of its block steps, with the panels (from the inverted
 *   diagonal blocks) and the trailing updates on tcgen05 tensor cores, three TF32 products
 *   per term (hi*hi + hi*lo + lo*hi, about 1.2e-6 relative error per product against 6e-8 for
 *   FP32; FP32 accumulation); the subdomain's trailing window stays in L2 between its steps. One launch per block step for
 *   the whole batch: 3 = tcgen05 with three TF32 products, 1 = one TF32 product, 4 = FP32
 *   CUDA cores. MX_PLAIN_FP64 always uses FP64 CUDA cores. */
#define MX_TUNE_LU_TENSOR 2
/*   MX_TUNE_COARSE_BLOCKS: thread blocks of the cooperative coarse sweep (0 = sized by the
 *   band work, at most one per SM); fewer blocks make its grid-wide barriers cheaper. */
#define MX_TUNE_COARSE_BLOCKS 3
/*   MX_TUNE_LOCAL_TENSOR: local solves of the MX_MIXED form; 1 = tcgen05 tensor cores
 *   (the off-diagonal band updates as TF32 GEMMs against panel images of the factors that
 *   mx_factor stores beside the band, about as many bytes again; the right-hand-side block
 *   enters as a TF32 hi + lo pair; default), 0 = FP32 CUDA-core substitution. Half-bandwidths
 *   above 448 fall back to the CUDA cores. Changing it after mx_factor builds the panel
 *   images at the next solve. */
#define MX_TUNE_LOCAL_TENSOR 4
/*   MX_TUNE_COARSE_INVERSE: coarse solve of the MX_MIXED form; 1 (default) = mx_factor
 *   forms the explicit c64 inverse of A^0 (n_c^2 complex entries, by band sweeps on the
 *   identity) and every apply is one dense product on the tcgen05 tensor cores (three TF32
 *   products per term; CUDA cores for an odd n_c), 2 = the same inverse with the product on
 *   the CUDA cores, 0 = band triangular sweeps. 0 takes effect at the next mx_factor. */
#define MX_TUNE_COARSE_INVERSE 5
/*   MX_TUNE_LU_GRID: CTAs of the persistent local LU (MX_TUNE_LU_TENSOR 0 or 2), each taking
 *   subdomains blockIdx, blockIdx + grid, ...; 0 (default) = one CTA per subdomain. A grid
 *   below the SM count keeps fewer trailing windows resident, so that they share L2. */
#define MX_TUNE_LU_GRID 6
/*   MX_TUNE_DOTS: second Gram-Schmidt pass of the MX_MIXED form (double-float inner
 *   products); 0 (default) = staged kernel (basis tiles of 8 vectors brought into a ring of
 *   shared-memory stages by bulk copies, one thread per row and pair of right-hand sides; 2, 4,
 *   8, 16 or 32 right-hand sides, otherwise the lane-parallel kernel), 1 = lane-parallel
 *   kernel. Same arithmetic per product, different summation order. */
#define MX_TUNE_DOTS 7
MX_API int mx_set_tuning(mx_handle h, int key, int value);

/* Preconditioner variant (Sec. 6.3), applied by mx_solve and mx_precond:
 *   MX_PREC_AS    additive Schwarz of Eq. 3.4 (default);
 *   MX_PREC_RAS   restricted additive Schwarz (Eq. RAS2): every DOF takes the local solution
 *                 of the subdomain that owns it (partition of unity D^l: the core box holding
 *                 the edge midpoint), plus the coarse term when there is a coarse level;
 *   MX_PREC_HRAS  hybrid two-level RAS (Eq. HRAS): (I - G A) B_RAS1^{-1} (I - A G) + G;
 *   MX_PREC_ADEF1 adapted deflation (Eq. ADEF1ras): B_RAS1^{-1} (I - A G) + G;
 * with G = (R^0)^T (A^0)^{-1} R^0 and A = A_{xi_prec}. The restricted variants need an
 * overlap of at least one cell (MX_EINVAL otherwise); HRAS and ADEF1 need a coarse level
 * and apply both levels whatever `levels` mx_precond gets. Takes effect at the next apply. */
#define MX_PREC_AS 0
#define MX_PREC_RAS 1
#define MX_PREC_HRAS 2
#define MX_PREC_ADEF1 3
MX_API int mx_set_preconditioner(mx_handle h, int kind);

/* Weighted GMRES (Sec. 5.2): 1 = the Arnoldi process and the residual minimisation of
 * mx_solve use the inner product <v, w>_D = w^H D_k v with D_k = K + k^2 M, the matrix of
 * the (.,.)_{curl,k} inner product (Eq. 5.1); the stopping test is then on
 * ||b - A x||_{D_k} / ||b||_{D_k} (true residual, FP64) and rel_residual reports that ratio.
 * Two products with D_k per iteration. 0 (default) = the Euclidean inner product. */
MX_API int mx_set_weighted_gmres(mx_handle h, int weighted);

/* Coarse solver of the two-level preconditioners (Sec. 6.4).
 *   MX_COARSE_DIRECT (default): the FP64 band LU of A^0 (and, in the mixed form, its
 *     explicit c64 inverse), built by mx_factor.
 *   MX_COARSE_GMRES: every coarse solve (A^0)^{-1} R^0 v is replaced by an inner
 *     right-preconditioned GMRES on A^0 y = R^0 v with y0 = 0, unrestarted, stopped at the
 *     relative Euclidean residual `tol` (0 < tol < 1; the paper takes 1e-1) or after
 *     `max_it` (1..1000) iterations, whichever comes first (a solution that misses tol is
 *     used as it is). Its preconditioner is one-level Schwarz, `prec_kind` MX_PREC_AS or
 *     MX_PREC_RAS, on subdomains of the coarse mesh described by `dd` (boxes of
 *     dd->core_cells coarse cells widened by dd->overlap_cells; RAS needs an overlap >= 1).
 *     The inner problem is built here with A^0 = K_c - (k^2 + i xi_prec) M_c and the
 *     handle's precision, and factored by mx_factor (or here, if the handle is already
 *     factored); the direct coarse factors are then not built. The outer GMRES of mx_solve
 *     keeps the preconditioned vectors z_j (flexible GMRES), so the varying inner solves
 *     are allowed.
 * MX_EINVAL for a handle without a coarse level or out-of-range arguments (the setting is
 * then unchanged). Switching back to MX_COARSE_DIRECT on a factored handle builds the
 * direct factors at once. */
#define MX_COARSE_DIRECT 0
#define MX_COARSE_GMRES 1
MX_API int mx_set_coarse_solver(mx_handle h, int kind, const mx_dd_desc* dd, double tol, int max_it, int prec_kind);

/* Message of the last error on the calling thread ("" if none). */
MX_API const char* mx_last_error(void);

/* Assemble the problem (Sec. 2.2, Eq. 2.2; Sec. 3, Eq. 3.1-3.3):
 * Kuhn mesh and edge numbering (PEC-interior edges, or all edges with the impedance
 * condition), CSR K and M (real FP64; and B with the impedance condition) with
 * A_xi = K - (k^2 + i xi) M [- i sign(xi) k B], subdomain index lists, and (two-level) the
 * coarse mesh, its Galerkin matrix A^0_{xi_prec} and the restriction R^0 of Eq. 3.2.
 * The preconditioner uses xi_prec, the operator xi_prob (Sec. 6.2).
 * Returns MX_EINVAL for n_cells < 1, core_cells < 1, overlap_cells < 0, k <= 0, an unknown
 * boundary, xi_prec == 0 with PEC (local matrices are only guaranteed invertible for
 * xi != 0, Sec. 3.3; the impedance local problems are well posed for xi = 0, as the
 * paper's Table 7 uses) or a coarse n_cells that does not divide the fine one. *out is
 * set on success only. */
MX_API int mx_build_problem(const mx_mesh_desc* mesh, double k, double xi_prob, double xi_prec,
                     const mx_dd_desc* dd, const mx_coarse_desc* coarse, int precision,
                     mx_handle* out);

/* Change xi_prob of the operator (the factors depend on xi_prec only). */
MX_API int mx_set_xi_prob(mx_handle h, double xi_prob);

/* Run all device work of this handle on the given cudaStream_t (NULL = legacy default). */
MX_API int mx_set_stream(mx_handle h, void* stream);

/* Factor the preconditioner (Eq. 3.3-3.4): extract every local minor
 * A^l = R^l A_{xi_prec} (R^l)^T and LU-factor all of them in one batch without
 * pivoting (coercivity, Lemma 2.2, keeps every pivot nonzero), c64 in MX_MIXED and c128
 * in MX_PLAIN_FP64; LU-factor the coarse matrix A^0 (band-limited; FP64 in MX_PLAIN_FP64,
 * c64 in MX_MIXED, which also forms the explicit inverse unless MX_TUNE_COARSE_INVERSE
 * is 0), or, with MX_COARSE_GMRES, factor the inner problem's subdomains instead.
 * Returns MX_ESINGULAR when a local or coarse pivot is zero or not finite, or when the
 * pivot growth of a local LU, max|U_ij| / max|A^l_ij|, exceeds the growth limit
 * (mx_set_growth_limit). Coercivity bounds the pivots away from zero but not the growth;
 * the factors carry relative errors of about the unit roundoff times the growth. The
 * largest growth is reported by mx_info. After MX_ESINGULAR or MX_ETIMEOUT the handle is
 * left unfactored: mx_solve and mx_precond return MX_ENOTFACTORED until an mx_factor
 * succeeds. */
MX_API int mx_factor(mx_handle h);

/* Pivot-growth limit of the local LU checked by mx_factor; limit <= 0 restores the default
 * (1e6 for the c64 factors of MX_MIXED, 1e12 for MX_PLAIN_FP64). Takes effect at the next
 * mx_factor. MX_EINVAL for a NaN limit. */
MX_API int mx_set_growth_limit(mx_handle h, double limit);

/* Load vectors f_i = int F . w_i (Sec. 2.2) for nrhs right-hand sides with
 * F(x) = sum_b pol_b exp(-|x - c_b|^2 / width^2):
 * centres [nrhs][nbumps][3] (host), pol [nrhs][nbumps][3] complex (host, interleaved),
 * f [nrhs][n_dof] c128 (host or device). Quadrature: conical-product Gauss-Legendre,
 * 3 points per direction, on every tetrahedron. */
MX_API int mx_load_vector(mx_handle h, int nrhs, int nbumps, const double* centres,
                   const double* pol, double width, void* f);

/* Solve A_{xi_prob} x = b for nrhs right-hand sides by right-preconditioned GMRES
 * (Sec. 6.1) with the additive Schwarz preconditioner B^{-1} of Eq. 3.4, restarted
 * every `restart` iterations (0 = unrestarted), x0 = 0, stopping per right-hand side when
 * the FP64 relative residual ||b - A x|| / ||b|| <= tol or after max_it iterations.
 * rhs, x: [nrhs][n_dof] c128, host or device. stats: nrhs entries (host) or NULL.
 * Returns MX_ENOCONV if any right-hand side did not converge (x is still the last
 * iterate). */
MX_API int mx_solve(mx_handle h, const void* rhs, int nrhs, double tol, int restart, int max_it,
             void* x, mx_rhs_stats* stats);

/* Number of unknowns (PEC-interior edges, or all edges with the impedance condition). */
MX_API int64_t mx_num_dofs(mx_handle h);

/* Sizes of the assembled problem. */
MX_API int mx_info(mx_handle h, mx_problem_info* out);

/* Device timings of the last build / factor / solve. */
MX_API int mx_timings(mx_handle h, mx_timing* out);

/* Free the handle and all its device memory. NULL is ignored. */
MX_API void mx_destroy(mx_handle h);

/* ---- Steps of the path, exposed for verification and composition ---------------- */

/* Integer mesh data (Sec. 2.2), host outputs:
 * dof_key [n_dof]: 7 * v_low + d of each DOF (v vertex id, d direction index),
 * tet2dof [6 n^3][6]: DOF of each local edge (01,02,03,12,13,23) of each tetrahedron,
 * -1 for PEC edges. Either pointer may be NULL. */
MX_API int mx_get_mesh(mx_handle h, int32_t* dof_key, int32_t* tet2dof);

/* Subdomain index sets I^h(Omega_l) (Eq. 3.1), host outputs: offsets [n_sub + 1],
 * lists [sum_local] (sorted global DOFs of each subdomain, concatenated);
 * inverse map inv_ptr [n_dof + 1], inv_pos [sum_local] (positions into `lists`, in
 * increasing subdomain order). Any pointer may be NULL. */
MX_API int mx_get_subdomains(mx_handle h, int64_t* offsets, int32_t* lists, int32_t* inv_ptr,
                      int32_t* inv_pos);

/* CSR of K and M (which = 0 fine, 1 coarse), host outputs rowptr [rows + 1],
 * col [nnz], K [nnz], M [nnz] (FP64). Any pointer may be NULL. */
MX_API int mx_get_csr(mx_handle h, int which, int32_t* rowptr, int32_t* col, double* K, double* M);

/* Values of the boundary mass B (Eq. imp) on the same CSR pattern as mx_get_csr (which = 0
 * fine, 1 coarse), host output B [nnz]; zeros for a PEC problem. */
MX_API int mx_get_boundary_mass(mx_handle h, int which, double* B);

/* R^0 of Eq. 3.2 as CSR [n_coarse x n_dof], host outputs. */
MX_API int mx_get_coarse_restriction(mx_handle h, int32_t* rowptr, int32_t* col, double* val);

/* y = A_{xi_prob} x (FP64), x and y [nrhs][n_dof] c128, host or device. */
MX_API int mx_spmv(mx_handle h, const void* x, void* y, int nrhs);

/* y = A_{xi_prob} x as the MX_MIXED Krylov process forms A z_j (Sec. 6.1, flexible GMRES):
 * x rounded to c64, each product and the sums of a row in double-float arithmetic (the
 * coefficients of K - (k^2 + i xi) M split into FP32 pairs), y the c128 value hi + lo of each
 * double-float result. Right-hand sides in pairs for an even nrhs, one at a time otherwise,
 * as in the solver. Same layouts as mx_spmv; any handle. For verification of that kernel. */
MX_API int mx_spmv_mixed(mx_handle h, const void* x, void* y, int nrhs);

/* z = B^{-1} v (Eq. 3.4) with the factored preconditioner; levels: bit 0 = local
 * solves (l >= 1), bit 1 = coarse solve (l = 0). v, z [nrhs][n_dof] c128. */
MX_API int mx_precond(mx_handle h, const void* v, void* z, int nrhs, int levels);

/* Copy the packed factor of subdomain l (after mx_factor) or its minor A^l (before),
 * column-major n_l x n_l, c128 (host). Unit lower L below the diagonal, U on and above. */
MX_API int mx_get_local(mx_handle h, int l, double* out);

/* Batched inner products of the Gram-Schmidt step of the Arnoldi process (Sec. 5.2 recalls
 * GMRES; the right-preconditioned GMRES of Sec. 6.1 orthogonalises each new vector
 * against the basis): h[i][r] = sum_x conj(V_i[x][r]) w[x][r] for i < nvec, r < nrhs.
 * V: nvec blocks [nvec][n][nrhs] c128 and w: [n][nrhs] c128, both device memory
 * (right-hand side index fastest); h: [nvec][nrhs] c128, host or device. FP64 products
 * and fixed-order reductions (deterministic). stream: a cudaStream_t (NULL = legacy default);
 * the call synchronises it. Scratch for the block partial sums is allocated per call
 * through the library's allocator. MX_EINVAL for nrhs outside 1..32, nvec < 1, n < 1 or
 * host V / w. */
MX_API int mx_dots(const void* V, const void* w, int64_t n, int nrhs, int nvec, void* h, void* stream);

/* mx_dots for callers that cannot allocate device memory: a host framework that owns all
 * device memory through its own pool and forbids side allocations (a cudaMalloc there
 * would bypass its accounting or fail under its fixed budget), or an embedding that has
 * no allocator to hand the library. The paper has no counterpart; it is a deployment
 * variant. Same arguments and layouts as mx_dots and the same results to rounding: the
 * block partial sums live in a fixed 4 MiB array inside the library's device image (held
 * on every GPU that loads the library until the process exits), so the call allocates
 * nothing; when nvec * nrhs is above about 860 the array holds fewer than 2 x SM-count
 * partial-sum blocks, so the summation order, and with it the last bits, depends on
 * nvec * nrhs. Limit: nvec * nrhs <= 16384, else MX_EINVAL with a message. The first call
 * on a device looks the array's device address up (cudaGetSymbolAddress, with that device
 * current) and keeps it for the life of the process, which assumes the device is not
 * reset (cudaDeviceReset) in between; make that first call before any stream capture.
 * Like mx_dots, the call synchronises `stream` before it returns. All calls on one device
 * share the array: calls that overlap on the GPU (unordered streams or threads) race on
 * it. Every word a call reads from the array is written earlier in the same call, so no
 * clearing is needed between calls. */
MX_API int mx_dots_noalloc(const void* V, const void* w, int64_t n, int nrhs, int nvec, void* h, void* stream);

/* Failure-path check (no counterpart in the paper): launches `blocks` blocks (1..1024) whose
 * first thread waits, with the same bounded mbarrier wait as the tensor-core kernels and a
 * limit of `limit` polls (1..2^20), on an mbarrier that nothing arrives on. Every wait runs
 * out, is counted in the handle's device error word and read back as the solves read it:
 * returns MX_ETIMEOUT, after which the handle and the CUDA context remain usable. The
 * probe holds no tensor memory and starts no copies. */
MX_API int mx_test_bounded_wait(mx_handle h, int limit, int blocks);

/* ---- Serving --------------------------------------------------------------------------
 * A request loop for many solves with different operators and right-hand-side counts on
 * one GPU. Worker threads (each with its own CUDA stream) take the oldest pending request
 * together with every pending request of the same operator and solver settings as one batch
 * of right-hand-side slots (twice the starting count rounded up to 8, at most 32). Continuous
 * batching: at every GMRES restart boundary of a running batch, requests whose right-hand
 * sides have all finished are returned at once, and pending requests of the same operator and
 * settings are admitted into free slots and solved in the same run (mx_server_info.joined
 * counts them); each slot keeps its own arithmetic, so a result does not depend on the
 * requests it was batched with. Batches of different operators run
 * concurrently. Factorisations stay resident in HBM, cached by the preconditioner key
 * (n_cells, k, xi_prec, subdomains, coarse mesh, precision, boundary condition,
 * preconditioner variant; xi_prob does not enter it, since
 * B^{-1} is built from A_{xi_prec} only, Sec. 6.2). A new factorisation is admitted when its
 * planned factor bytes plus the batch's Krylov workspace fit the budget after evicting idle
 * cached factorisations (least recently used first) and fit the device's free memory;
 * otherwise the batch waits, and while it waits no other batch starts and running batches
 * admit no new requests, so the memory they hold comes free within their iteration limits.
 * A waiting batch fails with MX_ENOMEM after 30 s in which no other batch held memory. */
typedef struct mx_server_s* mx_server;

typedef struct {
  int n_cells;             /* mesh (mx_mesh_desc) */
  double k, xi_prob, xi_prec;
  int core_cells, overlap_cells, coarse_cells, precision;
  int nrhs, nbumps;        /* right-hand sides as in mx_load_vector: 1..32 of them */
  const double* centres;   /* [nrhs][nbumps][3], copied at submit */
  const double* pol;       /* [nrhs][nbumps][3] complex, copied at submit */
  double width;
  double tol;              /* GMRES settings as in mx_solve */
  int restart, max_it;
  int boundary;            /* MX_BC_PEC or MX_BC_IMPEDANCE (mx_mesh_desc) */
  int prec_kind;           /* MX_PREC_AS, _RAS, _HRAS or _ADEF1 (mx_set_preconditioner) */
} mx_request;

typedef struct {
  double latency_ms;       /* submit -> result available, host clock */
  double queue_ms;         /* submit -> start of the batch that solved it */
  int64_t n_dof;
} mx_request_timing;

typedef struct {
  int64_t batches;         /* batches started */
  int64_t factorisations, evictions, completed, cached_bytes;
  int32_t cached_operators, pending;
  int64_t joined;          /* requests admitted into a batch that was already running */
  int32_t waiting_for_memory; /* batches waiting for their factorisation to fit the budget */
} mx_server_info;

#define MX_PENDING 1       /* mx_server_poll without wait: result not ready yet */

/* Start a server with a device memory budget for cached factorisations and workspaces,
 * and `workers` worker threads / streams (1..16). */
MX_API int mx_server_create(int64_t budget_bytes, int workers, mx_server* out);
/* Queue a request; returns a ticket. Arrays are copied before the call returns. */
MX_API int mx_server_submit(mx_server s, const mx_request* req, int64_t* ticket);
/* Result of a ticket: with wait = 0 returns MX_PENDING if not finished; otherwise blocks.
 * x: [nrhs][n_dof] c128 host (or NULL), stats: nrhs entries (or NULL), timing (or NULL).
 * Returns the request's MX_OK / MX_ENOCONV / error code and forgets the ticket. */
MX_API int mx_server_poll(mx_server s, int64_t ticket, int wait, void* x, mx_rhs_stats* stats,
                          mx_request_timing* timing);
MX_API int mx_server_stats(mx_server s, mx_server_info* out);
/* Finish running batches, stop the workers and free every cached factorisation. Pending
 * requests that were not started are dropped. */
MX_API void mx_server_destroy(mx_server s);

/* ---- Instrumentation ----------------------------------------------------------------- */

/* Number of kernel launches made by the library since it was loaded (all handles). */
MX_API int64_t mx_launch_count(void);

/* Enable (1) or disable (0) per-kernel device timing and clear the accumulators. When
 * enabled, each step of the path is bracketed by CUDA events on the handle's stream;
 * the events add about a microsecond of host time per step. */
MX_API int mx_profile(int enable);

/* Resolve pending events (synchronises) and copy, per kernel id, the accumulated device
 * milliseconds, launches, algorithmic bytes and flops (any pointer may be NULL; arrays
 * hold at least the returned count of entries). Returns the number of kernel ids. */
MX_API int mx_profile_read(double* ms, int64_t* launches, double* bytes, double* flops);

/* Name of kernel id `id` ("" if out of range). */
MX_API const char* mx_profile_name(int id);

#ifdef __cplusplus
}
#endif

#endif /* MXAS_H */

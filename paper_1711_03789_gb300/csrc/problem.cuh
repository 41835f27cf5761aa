// Internal state of one assembled problem and the declarations of the kernels'
// host launchers, grouped by step of the path.
#pragma once

#include "common.cuh"

namespace mx {

// Kuhn mesh of the unit cube with n cells per side and its PEC-interior edge DOFs
// (Sec. 2.2). Edge (v, d) runs from vertex v to v + DIRS[d]; its key is 7 v + d.
struct MeshDev {
  int n = 0;
  int64_t n_dof = 0;
  DevBuf<int32_t> edge_dof;  // [(n+1)^3 * 7]  DOF of edge key, -1 if PEC or absent
  DevBuf<int32_t> dof_key;   // [n_dof]
  DevBuf<int32_t> tet2dof;   // [6 n^3 * 6]
};

// Real CSR with the curl-curl (K) and mass (M) values on one pattern, and the tangential
// boundary mass (B) of the impedance condition (empty with PEC).
struct CsrKM {
  int64_t rows = 0, cols = 0, nnz = 0;
  DevBuf<int32_t> rowptr, col;
  DevBuf<double> K, M, B;
};

// Plain CSR with one real value per entry (R^0 and its transpose).
struct CsrR {
  int64_t rows = 0, cols = 0, nnz = 0;
  DevBuf<int32_t> rowptr, col;
  DevBuf<double> val;
};

struct Timing {
  double build_ms = 0, factor_ms = 0, solve_ms = 0;
  int64_t solve_launches = 0;
  int restarts = 0, max_iterations = 0;
  int64_t coarse_inner_iterations = 0, coarse_inner_solves = 0;
};

struct Workspace;  // solve buffers (krylov.cu)

// A batch of band matrices (LAPACK band layout, see local.cu).
constexpr int LU_NB = 32;
struct BandBatch {
  int count;
  const int32_t* n;    // [count]
  const int32_t* b;    // [count] half-bandwidth
  const int32_t* ld;   // [count] leading dimension (>= 2 b + 1)
  const int64_t* off;  // [count] element offsets
  uint32_t* umax;      // [count] largest |U_ij| met by the factorisation, as FP32 bits (or null)
};

__host__ __device__ inline int64_t bidx(int64_t off, int ld, int b, int i, int j) {
  return off + (int64_t)j * ld + (b + i - j);
}

struct Problem {
  // parameters
  int n = 0, core = 0, overlap = 0, coarse_m = 0, precision = MX_MIXED;
  int bc = MX_BC_PEC;  // MX_BC_IMPEDANCE: all edges are DOFs, ImpRAS local problems
  double k = 0, xi_prob = 0, xi_prec = 0;
  cudaStream_t stream = nullptr;

  // fine and coarse meshes and matrices
  MeshDev fine, coarse;
  CsrKM A, Ac;  // A_xi = K - (k^2 + i xi) M

  // subdomains (Eq. 3.1): boxes, sorted index lists, inverse map DOF -> positions
  int n_sub = 0, n_per_axis = 0;
  std::vector<int32_t> box;        // [n_sub][6] lo xyz, hi xyz (vertex indices)
  std::vector<int64_t> h_offsets;  // [n_sub + 1]
  std::vector<int32_t> h_nl;       // [n_sub]
  int max_local = 0;
  int64_t sum_local = 0;
  DevBuf<int64_t> offsets;         // [n_sub + 1]
  DevBuf<int32_t> nl;              // [n_sub]
  DevBuf<int32_t> lists;           // [sum_local]
  DevBuf<int32_t> inv_ptr;         // [n_dof + 1]
  DevBuf<int32_t> inv_pos;         // [sum_local]
  // preconditioner variant (Sec. 6.3): MX_PREC_AS, MX_PREC_RAS, MX_PREC_HRAS, MX_PREC_ADEF1;
  // the restricted ones scatter only the owner's local solution of every DOF
  int prec_kind = MX_PREC_AS;
  DevBuf<int32_t> own_pos;         // [n_dof] position of the DOF in its owner's list

  // local factors: band storage (see local.cu), element type float2 (mixed) or double2
  // (plain), matrix l at mat_off[l] elements.
  bool dense_local = false;        // force b_l = n_l - 1 (full dense storage)
  int tune_local_group = 0;        // cap on right-hand sides per local-solve block (0 = 16)
  int tune_lu_grid = 0;            // CTAs of the persistent LU (0: one per subdomain)
  int tune_dots = 0;               // second Gram-Schmidt pass (mixed): 0 staged, 1 lane-parallel
  int tune_lu_tc = 0;              // FP32 local LU: 0 / 2 persistent 3 x TF32 tensor-core LU, per-step
                                   // launches with 1 TF32 or 3 split 3 x TF32 tensor-core updates, 4 FP32 CUDA cores
  int tune_coarse_blocks = 0;      // blocks of the cooperative coarse sweep (0 = by work)
  std::vector<int32_t> h_band;     // [n_sub] half-bandwidths
  int64_t band_entries = 0;        // sum over subdomains of entries with |i - j| <= b_l
  DevBuf<int32_t> band;
  std::vector<int64_t> h_mat_off;  // [n_sub + 1]
  std::vector<int32_t> h_ld;
  DevBuf<int64_t> mat_off;
  DevBuf<int32_t> ld;
  DevBuf<unsigned char> factors;
  DevBuf<int64_t> dinv_off;        // [n_sub + 1] offsets of the inverted diagonal blocks
  DevBuf<unsigned char> dinv;      // inverted NB x NB diagonal blocks of L and U
  // tensor-core local solves (mixed form): TF32-rounded panel images of the factors in the
  // K-major shared-memory layout, one per block column and sweep (local_tc.cu)
  int tune_local_tc = 1;           // 0 CUDA-core substitution, 1 tensor-core panels (mixed form)
  bool panels_ok = false;
  int64_t panel_bytes = 0;
  DevBuf<unsigned char> panels;
  DevBuf<int64_t> pan_start;       // [n_sub + 1] first panel of each subdomain
  DevBuf<int64_t> pan_tab;         // byte offset of every panel image
  bool factored = false;
  bool minors_ready = false;

  // coarse space (Eq. 3.2): R^0 [n_c x n], its transpose, dense A^0 and its LU (FP64),
  // and a c64 copy of the factors for the mixed-precision coarse solve.
  CsrR R0, R0T;
  DevBuf<float> R0T_valf;  // FP32 copy of the R^0^T values (mixed-form scatter)
  DevBuf<float> R0_valf;   // FP32 copy of the R^0 values (mixed-form coarse restriction)
  // mixed-form operator coefficients a + i b = K - (k^2 + i xi_prob) M as double-floats
  DevBuf<float4> A_coef_df[3];     // 0: xi_prob (operator), 1: xi_prec (hybrid preconditioners), 2: D_k
  double A_coef_xi[3] = {-1.0, -1.0, -1.0};
  bool weighted = false;           // weighted GMRES in the D_k = K + k^2 M inner product (Sec. 5.2)
  int64_t n_c = 0;
  int coarse_band = 0;
  int64_t ld_c = 0;
  DevBuf<double2> A0;     // band storage [n_c * ld_c], LU in place after factor
  DevBuf<float2> A0f;     // c64 copy of the factors (mixed)
  DevBuf<int32_t> c_meta; // n, b, ld of the coarse band matrix (device)
  DevBuf<int64_t> c_off;
  DevBuf<double2> c_dinv; // inverted diagonal blocks of the coarse factors (FP64)
  DevBuf<float2> c_dinvf; // c64 copy (mixed)
  // mixed form: the explicit c64 inverse of A^0 (row-major; A^0 is complex symmetric, so
  // is its inverse), applied as one dense product instead of the band sweeps
  int tune_coarse_inverse = 1;     // used while n_c <= COARSE_INVERSE_MAX and the band fits the solve window
  DevBuf<float2> A0inv;
  DevBuf<float2> c_part;  // split-K partial products of the dense coarse apply
  DevBuf<int32_t> status; // [4] device error words: 0 local pivot, 1 coarse pivot, 2 timeout
  // pivot growth of the local LU: largest |A^l_ij| and |U_ij| per subdomain (FP32 bits)
  DevBuf<uint32_t> amax, umax;
  double growth_limit = 0;   // 0: default (1e6 for c64 factors, 1e12 for c128)
  double max_growth = 0;     // max over subdomains of max|U| / max|A^l| after the last factor
  int growth_worst = -1;     // the subdomain that reached it
  bool coarse_factored = false;  // direct coarse factors built
  // inexact coarse solve (Sec. 6.4): an inner GMRES on A^0 y = R^0 v, preconditioned by
  // one-level Schwarz on subdomains of the coarse mesh -- a problem of its own, built on
  // the coarse mesh with xi_prob = xi_prec of this one
  Problem* coarse_inner = nullptr;
  double c_tol = 0.1;
  int c_max_it = 100;
  DevBuf<double2> c_rhs, c_sol;  // [n_c][nrhs] R^0 v and the inner solution (FP64)

  Workspace* ws = nullptr;
  Timing timing;

  ~Problem();
};

// the explicit c64 coarse inverse is formed for coarse problems up to this size (n_c^2 c64
// entries: 2.1 GB); larger coarse problems keep the band sweeps
constexpr int64_t COARSE_INVERSE_MAX = 16384;

// ---- api.cu -------------------------------------------------------------------------
// validate, build mesh / assembly / subdomains / coarse space on `stream` (throws Error)
Problem* create_problem(int n, double k, double xi_prob, double xi_prec, int core, int overlap, int coarse_m,
                        int precision, cudaStream_t stream, int bc = MX_BC_PEC);
// extract minors, batched local LU, coarse LU; checks pivots and waits (throws Error)
void factor_problem(Problem& P);
// device bytes of the local factors a factorisation will allocate (runs the band pass)
int64_t local_factor_bytes(Problem& P);
// [nrhs][n] (caller layout) <-> [n][nrhs] (solver layout), device to device
void transpose_to_internal(const double2* user, double2* in, int64_t n, int nrhs, cudaStream_t s);
void transpose_to_user(const double2* in, double2* user, int64_t n, int nrhs, cudaStream_t s);

// ---- mesh.cu ------------------------------------------------------------------------
// all_edges: every edge is a DOF (impedance condition), else the PEC-interior ones
void build_mesh(MeshDev& m, int n, cudaStream_t s, bool all_edges = false);
void build_subdomains(Problem& P);
// owner positions of the partition of unity of the restricted variants (once)
void build_owner(Problem& P);

// ---- assemble.cu --------------------------------------------------------------------
// boundary: also B, the tangential mass of the boundary triangles (impedance condition)
void assemble_KM(const MeshDev& m, CsrKM& A, cudaStream_t s, bool boundary = false);
// ImpRAS local matrices (Sec. 6.3): K - (k^2 + i xi_prec) M - i sign(xi_prec) k B of every
// closed subdomain box (tetrahedra inside the box, triangles on its surface) into the
// band storage of the local factors (element type of the precision)
void extract_imp(Problem& P);
// coefficient c of the impedance term -i c B of A_xi: sign(xi) k (sign(0) = +1), 0 for PEC
inline double imp_coef(const Problem& P, double xi) {
  return P.bc == MX_BC_IMPEDANCE ? (xi < 0 ? -P.k : P.k) : 0.0;
}
void load_vector(const Problem& P, int nrhs, int nbumps, const double* h_centres,
                 const double* h_pol, double width, double2* f /* [nrhs][n] device */);
void build_coarse_restriction(Problem& P);

// ---- local.cu -----------------------------------------------------------------------
void extract_minors(Problem& P);
void factor_local(Problem& P);
// factor_local in two halves: queue the LU (async), then wait and build the panel images
void factor_local_launch(Problem& P);
void factor_local_finish(Problem& P);
template <typename T2>
void band_lu(const BandBatch& B, T2* A, int max_n, int max_span, int32_t* status, cudaStream_t s,
             const int32_t* hn, const int32_t* hb, int kid_update, int tc_split);
// one tcgen05 trailing-update step of the FP32 band LU (lu_tc.cu); split 1 or 3 TF32 products
void lu_update_tc(const BandBatch& B, float2* A, int k0, int max_span, int split, int32_t* status, cudaStream_t s);
// the whole FP32 band LU of every matrix of the batch in one persistent launch, one CTA per
// matrix, tcgen05 trailing updates (lu_fused.cu); bytes / flops: algorithmic, for the profiler
// also writes the inverted diagonal blocks (dinv at doff, as invert_diag_blocks does); needs
// every half-bandwidth within band_lu_fused_fits
void band_lu_fused(const BandBatch& B, float2* A, const int64_t* doff, float2* dinv, int split, int grid,
                   int32_t* status, cudaStream_t s, double bytes, double flops);
bool band_lu_fused_fits(int max_span);
template <typename T2>
void invert_diag_blocks(const BandBatch& B, const T2* A, const int64_t* doff, T2* Dinv, int max_n, cudaStream_t s);
// z_l = (A^l)^{-1} R^l v for every l, written at the subdomain positions of `loc`
// (element type of the factors), v [n][nrhs] c128 (vtype 0), c64 (1) or complex
// double-float (3, whose c64 rounding is its high half).
void local_solves(Problem& P, const void* v, int vtype, void* loc, int nrhs);
// X = (A^0)^{-1} from the c64 coarse band factors (row-major n_c x n_c, c64)
void coarse_inverse(Problem& P, float2* X);

// ---- coarse_tc.cu -------------------------------------------------------------------
// part[ks][i][r] = split ks of sum_j X[i][j] rin[j][r] on the tensor cores (3 x TF32), X the
// explicit c64 coarse inverse; sets the split count. false (nothing launched) for an odd n_c.
bool coarse_dense_tc(Problem& P, const float2* rin, int nrhs, float2*& part, int& ks);

// ---- local_tc.cu --------------------------------------------------------------------
// panel images of the c64 factors for the tensor-core solves (after factor_local)
void build_panels(Problem& P);
// bytes build_panels will allocate (0 when a half-bandwidth is too large for them)
int64_t panel_bytes_planned(const Problem& P);
// the local solves of local_solves() on the tensor cores (requires P.panels_ok)
void local_solves_tc(Problem& P, const void* v, int vtype, void* loc, int nrhs, double alg_bytes, double alg_flops);
// bounded waits on an mbarrier nothing arrives on, in `blocks` blocks; returns how many ran
// out (read back through status[2], as after the local solves)
int32_t wait_probe(Problem& P, int limit, int blocks);

// ---- coarse.cu ----------------------------------------------------------------------
void factor_coarse(Problem& P);
// y = (A^0)^{-1} R^0 v: coarse_rhs [nrhs][n_c] c128 workspace
void coarse_solve(Problem& P, const void* v, int vtype, double2* yc, int nrhs);

// ---- krylov.cu ----------------------------------------------------------------------
// y = A_{xi} x; x c128 or c64 [nrhs][n] (xtype 0/1), y c128
void spmv(const Problem& P, double xi, const void* x, int xtype, double2* y, int nrhs,
          cudaStream_t s);
// z = B^{-1} v into z [nrhs][n] c128 (ztype 0) or c64 (ztype 1); v c128 (vtype 0) or
// complex double-float (vtype 3, float4 {re_hi, im_hi, re_lo, im_lo})
void precond_apply(Problem& P, const void* v, void* z, int ztype, int nrhs, int levels, double2* zc = nullptr,
                   int vtype = 0);
// Restart-boundary hook of gmres_solve (continuous batching in the server). At every restart
// boundary the solver reports the columns that finished since the last call (their x in x_dev,
// internal [n][nrhs] layout, is final; its / rel / est hold their statistics); the hook returns
// the columns into which it wrote new right-hand sides (b_dev, same layout), which then start
// from x = 0 with their own ||b|| and iteration count. Columns keep their own arithmetic, so a
// right-hand side gets the same iterates whichever columns it shares the batch with.
struct SlotHook {
  virtual ~SlotHook() = default;
  virtual std::vector<int> at_restart(const double2* x_dev, double2* b_dev, const std::vector<int>& finished,
                                      const std::vector<int32_t>& its, const std::vector<double>& rel,
                                      const std::vector<double>& est) = 0;
};
int gmres_solve(Problem& P, const double2* b, double2* x, int nrhs, double tol, int restart,
                int max_it, mx_rhs_stats* stats, SlotHook* hook = nullptr);
void free_workspace(Problem& P);

// ---- krylov_df.cu: double-float Krylov kernels of the mixed form --------------------
void spmv_df(Problem& P, const float2* z, float4* w, int nrhs, cudaStream_t s);
// conversions around spmv_df for verification: c128 -> c64 (nearest), double-float -> c128
void c128_to_c64(const double2* a, float2* b, int64_t count, cudaStream_t s);
void df_to_c128(const float4* w, double2* y, int64_t count, cudaStream_t s);
// y = A_xi z, z c64, y c128 (double-float accumulation)
void spmv_df_c128(Problem& P, double xi, const float2* z, double2* y, int nrhs, cudaStream_t s);
// The basis of the mixed form is two c64 planes: Vh [m+1][n][nrhs] (c64 rounding) and Vl
// (remainder); vector i at offset i * n * nrhs of each.
// Block partials go to hpart[b][i][r] for b < the returned block count (at most nblk). Given
// `timeout` (a device counter; null selects the lane-parallel kernels), no `extra` and no norm
// entry, nrhs of 2, 4, 8, 16 or 32 takes the staged kernel, whose bounded waits count into *timeout.
int dots_df(int nblk, int64_t n, int nrhs, int nvec, int with_norm, const float2* Vh, const float2* Vl,
            const float4* w, const int32_t* active, double2* hpart, cudaStream_t s, const float4* extra = nullptr,
            int32_t* timeout = nullptr);
// first Gram-Schmidt pass: FP32 products of the c64 planes, FP64 partials
void dots_c64(int nblk, int64_t n, int nrhs, int nvec, const float2* Vh, const float4* w, const int32_t* active,
              double2* hpart, cudaStream_t s);
// v_{j+1} = (w' - Vh g) inv into the planes (g: c64 pass-2 coefficients, inv: 1/||w''|| split)
void update2_normalize(int64_t nv, int nrhs, int nvec, const float2* Vh, const float2* g, const float2* inv,
                       const float4* w, float2* vh, float2* vl, cudaStream_t s);
// x += Z y over the first kcols[r] columns (kmax the largest), Z c64, y FP64 (split into ys)
void update_x_df(int64_t nv, int nrhs, int kmax, const int32_t* kcols, const float2* Z, const double2* y, float4* ys,
                 double2* x, cudaStream_t s);
// y = D_k w, D_k = K + k^2 M, double-float vectors
void dmul_df(Problem& P, const float4* w, float4* y, int nrhs, cudaStream_t s);
void orth_update_df(int nblk, int64_t n, int nrhs, int nvec, const float2* Vh, const float2* Vl, const double2* h,
                    float4* hs, const int32_t* active, float4* w, double* npart, cudaStream_t s);
void normalize_df(int64_t nv, int nrhs, int j, int m, const double2* H, const int32_t* active, const float4* w,
                  float2* vh, float2* vl, cudaStream_t s);
void scale_v0_df(int64_t nv, int nrhs, const double* beta, const int32_t* active, const double2* r, float2* vh,
                 float2* vl, cudaStream_t s);
// h[i][r] = sum_x conj(V_i[x][r]) w[x][r], i < nvec; V [nvec][n][nrhs], w [n][nrhs] (device);
// partials: nblk * nvec * nrhs entries of scratch; ones: nrhs flags equal to 1
void batched_dots(const double2* V, const double2* w, int64_t n, int nrhs, int nvec, double2* h, double2* partials,
                  int nblk, const int32_t* ones, cudaStream_t s);
void fill_i32(int32_t* p, int n, int32_t v, cudaStream_t s);

}  // namespace mx

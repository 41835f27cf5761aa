// Operator, preconditioner apply and batched right-preconditioned GMRES (Sec. 6.1).
//
// Vectors inside the solver are stored [n][nrhs] (right-hand side index fastest) so the
// gathers of the SpMV, the restriction and the scatter read one contiguous segment per
// DOF. The right-preconditioned iteration is run in its flexible form: z_j = B^{-1} v_j is
// stored (c64 in MX_MIXED, c128 in MX_PLAIN_FP64), w = A z_j is formed in FP64, so the
// Arnoldi relation A Z_m = V_{m+1} H_m holds for the stored z_j whatever the precision
// of the preconditioner; x = x0 + Z_m y. Arnoldi is classical Gram-Schmidt with a second
// pass when the norm drops below 1/sqrt(2) of its value before orthogonalisation
// (Daniel-Gragg-Kaufman-Stewart criterion), in FP64 with fixed-order reductions. The
// least-squares problem is updated by complex Givens rotations; the stopping test uses
// the FP64 true residual ||b - A x|| / ||b|| at every restart and at the end.
#include "problem.cuh"

#include <algorithm>
#include <cmath>

namespace mx {

// ---- SpMV ---------------------------------------------------------------------------
// y[i][r] = sum_e (K_e - s M_e - i bc B_e) x[col_e][r],  s = k^2 + i xi (B: impedance term,
// absent with PEC)
template <typename XT>
__global__ void k_spmv(int64_t rows, int nrhs, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ K, const double* __restrict__ M, double sr, double si,
                       const XT* __restrict__ x, double2* __restrict__ y, const double* __restrict__ B, double bc) {
  const int64_t work = rows * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const int64_t i = t / nrhs;
    double2 kx = make_double2(0, 0), mx_ = make_double2(0, 0);
    const int32_t e1 = rowptr[i + 1];
    for (int32_t e = rowptr[i]; e < e1; ++e) {
      const double2 xv = to_c128(x[(int64_t)col[e] * nrhs + r]);
      const double k = K[e], m = M[e];
      kx.x = fma(k, xv.x, kx.x);
      kx.y = fma(k, xv.y, kx.y);
      mx_.x = fma(m, xv.x, mx_.x);
      mx_.y = fma(m, xv.y, mx_.y);
    }
    // K x - (sr + i si) M x
    double2 out = make_double2(kx.x - sr * mx_.x + si * mx_.y, kx.y - sr * mx_.y - si * mx_.x);
    if (B) {  // - i bc B x
      double2 bx = make_double2(0, 0);
      for (int32_t e = rowptr[i]; e < e1; ++e) {
        const double b = B[e];
        if (b == 0.0) continue;
        const double2 xv = to_c128(x[(int64_t)col[e] * nrhs + r]);
        bx.x = fma(b, xv.x, bx.x);
        bx.y = fma(b, xv.y, bx.y);
      }
      out.x += bc * bx.y;
      out.y -= bc * bx.x;
    }
    y[t] = out;
  }
}

static void spmv_km(const Problem& P, double sr, double si, const void* x, int xtype, double2* y, int nrhs,
                    cudaStream_t s, double bc = 0.0);

void spmv(const Problem& P, double xi, const void* x, int xtype, double2* y, int nrhs, cudaStream_t s) {
  spmv_km(P, P.k * P.k, xi, x, xtype, y, nrhs, s, imp_coef(P, xi));
}

// y = (K - (sr + i si) M - i bc B) x (bc = 0: no boundary term)
static void spmv_km(const Problem& P, double sr, double si, const void* x, int xtype, double2* y, int nrhs,
                    cudaStream_t s, double bc) {
  const double* B = (bc != 0.0 && P.A.B.p) ? P.A.B.p : nullptr;
  const int64_t work = P.A.rows * nrhs;
  // K, M values and column indices once, x once, y once (algorithmic minimum)
  const double xb = xtype == 0 ? 16.0 : 8.0;
  ProfScope ps(K_SPMV, s, 1, 20.0 * P.A.nnz + 4.0 * (P.A.rows + 1) + (xb + 16.0) * (double)P.A.rows * nrhs,
               8.0 * (double)P.A.nnz * nrhs);
  if (xtype == 0)
    MX_LAUNCH(k_spmv<double2><<<grid_for(work, 256, 152LL * 32), 256, 0, s>>>(P.A.rows, nrhs, P.A.rowptr.p, P.A.col.p, P.A.K.p,
                                                                    P.A.M.p, sr, si, (const double2*)x, y, B, bc));
  else
    MX_LAUNCH(k_spmv<float2><<<grid_for(work, 256, 152LL * 32), 256, 0, s>>>(P.A.rows, nrhs, P.A.rowptr.p, P.A.col.p, P.A.K.p,
                                                                   P.A.M.p, sr, si, (const float2*)x, y, B, bc));
  MX_CHECK_LAUNCH();
}

// ---- preconditioner: scatter-add of local solutions (+ coarse prolongation) ---------
// z[i][r] = sum_{q in inv(i)} loc[q][r] + sum_{p} (R^0)^T_{ip} y0[p][r]   (Eq. 3.4)
// zc (optional): the stored z promoted to c128, so that the operator reads exactly the
// stored vector without converting it once per nonzero.
template <typename T2> __device__ inline T2 cvt2(float2 a);
template <> __device__ inline float2 cvt2<float2>(float2 a) { return a; }
template <> __device__ inline double2 cvt2<double2>(float2 a) { return to_c128(a); }
template <typename T2> __device__ inline T2 cvt2(double2 a) { return conv<T2>(a); }

// Accumulation in AT: FP32 for the mixed form, whose z is stored in c64 anyway; FP64
// otherwise. The local solutions are summed in the fixed order of the inverse map.
template <typename LT, typename CT, typename ZT, typename AT>
__global__ void k_scatter(int64_t n, int nrhs, const int32_t* __restrict__ inv_ptr, const int32_t* __restrict__ inv_pos,
                          const int32_t* __restrict__ own, const LT* __restrict__ loc,
                          const int32_t* __restrict__ tptr, const int32_t* __restrict__ tcol,
                          const AT* __restrict__ tval, const CT* __restrict__ y0, int use_local, ZT* __restrict__ z,
                          double2* __restrict__ zc) {
  using A2 = typename cplx<AT>::type;
  const int64_t work = n * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const int64_t i = t / nrhs;
    A2 acc = czero<A2>();
    if (use_local && own) {
      acc = cvt2<A2>(loc[(int64_t)own[i] * nrhs + r]);  // restricted: the owner's solution only
    } else if (use_local)
      for (int32_t q = inv_ptr[i]; q < inv_ptr[i + 1]; ++q) {
        const int32_t pos = inv_pos[q];
        if (pos < 0) continue;
        const A2 v = cvt2<A2>(loc[(int64_t)pos * nrhs + r]);
        acc.x += v.x;
        acc.y += v.y;
      }
    if (tptr)
      for (int32_t e = tptr[i]; e < tptr[i + 1]; ++e) {
        const A2 v = cvt2<A2>(y0[(int64_t)tcol[e] * nrhs + r]);
        acc.x = fma(tval[e], v.x, acc.x);
        acc.y = fma(tval[e], v.y, acc.y);
      }
    const ZT zv = cvt2<ZT>(acc);
    z[t] = zv;
    if (zc) zc[t] = to_c128(zv);
  }
}

// The mixed form with an even number of right-hand sides: one thread per (DOF, pair of
// right-hand sides) with 16-byte loads of the c64 local and coarse solutions. The first 8
// inverse-map positions and the first 8 entries of the DOF's R^0 column are fetched before the
// loads that depend on them, so those loads are in flight together (a DOF lies in at most 8
// boxes when the overlap is below the core size; the loops continue past 8 otherwise). Same
// order of summation as k_scatter.
template <typename ZT>
__global__ void k_scatter2(int64_t n, int nrhs, const int32_t* __restrict__ inv_ptr, const int32_t* __restrict__ inv_pos,
                           const int32_t* __restrict__ own, const float4* __restrict__ loc,
                           const int32_t* __restrict__ tptr, const int32_t* __restrict__ tcol,
                           const float* __restrict__ tval, const float4* __restrict__ y0, int use_local,
                           ZT* __restrict__ z, double2* __restrict__ zc) {
  const int half = nrhs / 2;
  const int64_t work = n * half;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r2 = (int)(t % half);
    const int64_t i = t / half;
    float4 acc = zero;  // (re, im) of right-hand sides 2 r2 and 2 r2 + 1
    if (use_local && own) {
      acc = loc[(int64_t)own[i] * half + r2];  // restricted: the owner's solution only
    } else if (use_local) {
      const int32_t q0 = inv_ptr[i], q1 = inv_ptr[i + 1];
      int32_t pos[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) pos[k] = q0 + k < q1 ? inv_pos[q0 + k] : -1;
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = pos[k] >= 0 ? loc[(int64_t)pos[k] * half + r2] : zero;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (pos[k] >= 0) {
          acc.x += v[k].x;
          acc.y += v[k].y;
          acc.z += v[k].z;
          acc.w += v[k].w;
        }
      for (int32_t q = q0 + 8; q < q1; ++q) {
        const int32_t p = inv_pos[q];
        if (p < 0) continue;
        const float4 u = loc[(int64_t)p * half + r2];
        acc.x += u.x;
        acc.y += u.y;
        acc.z += u.z;
        acc.w += u.w;
      }
    }
    if (tptr) {
      const int32_t e0 = tptr[i], e1 = tptr[i + 1];
      int32_t c[8];
      float w[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        c[k] = e0 + k < e1 ? tcol[e0 + k] : -1;
        w[k] = e0 + k < e1 ? tval[e0 + k] : 0.f;
      }
      float4 y[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) y[k] = c[k] >= 0 ? y0[(int64_t)c[k] * half + r2] : zero;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (c[k] >= 0) {
          acc.x = fmaf(w[k], y[k].x, acc.x);
          acc.y = fmaf(w[k], y[k].y, acc.y);
          acc.z = fmaf(w[k], y[k].z, acc.z);
          acc.w = fmaf(w[k], y[k].w, acc.w);
        }
      for (int32_t e = e0 + 8; e < e1; ++e) {
        const float4 u = y0[(int64_t)tcol[e] * half + r2];
        const float wv = tval[e];
        acc.x = fmaf(wv, u.x, acc.x);
        acc.y = fmaf(wv, u.y, acc.y);
        acc.z = fmaf(wv, u.z, acc.z);
        acc.w = fmaf(wv, u.w, acc.w);
      }
    }
    const int64_t o = i * nrhs + 2 * r2;
    const ZT za = cvt2<ZT>(make_float2(acc.x, acc.y)), zb = cvt2<ZT>(make_float2(acc.z, acc.w));
    z[o] = za;
    z[o + 1] = zb;
    if (zc) {
      zc[o] = to_c128(za);
      zc[o + 1] = to_c128(zb);
    }
  }
}

__global__ void k_to_f32(int64_t n, const double* a, float* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

struct Workspace {
  int nrhs = 0, m = 0;
  int64_t n = 0;
  size_t zsz = 0;
  DevBuf<double2> V;              // (m+1) [n][nrhs]
  DevBuf<unsigned char> Z;        // m [n][nrhs] of c64 / c128
  DevBuf<double2> w, b, x, r;     // [n][nrhs]
  DevBuf<double2> zc;             // [n][nrhs] current z_j promoted to c128 (unused by the solver)
  DevBuf<float4> hs;              // [m+2][nrhs] h of the current pass as double-floats (mixed)
  DevBuf<float2> g2;              // [m+1][nrhs] pass-2 coefficients rounded to c64 (mixed)
  DevBuf<float2> inv2;            // [nrhs] 1 / ||w''|| as a double-float (mixed)
  DevBuf<double2> pv;             // 3 [n][nrhs] work vectors of the hybrid preconditioners
  DevBuf<unsigned char> loc;      // [sum_local][nrhs] local solutions
  DevBuf<double2> yc;             // [n_c][nrhs]
  DevBuf<double2> H;              // [m][m+1][nrhs]   column j, row i
  DevBuf<double> cs;              // [m][nrhs]
  DevBuf<double2> sn;             // [m][nrhs]
  DevBuf<double2> g;              // [m+1][nrhs]
  DevBuf<double2> y;              // [m][nrhs]
  DevBuf<double2> hpart;          // [nblk][m+2][nrhs] partial dot products
  DevBuf<double2> h2;             // [m+2][nrhs] reduced dots of the current pass
  DevBuf<double2> h1;             // [m+2][nrhs] first-pass dots (weighted Arnoldi)
  DevBuf<double> npart;           // [nblk][nrhs]
  DevBuf<double> bnorm, wnorm0;   // [nrhs]
  DevBuf<int32_t> active;         // [nrhs] 1 while the right-hand side iterates
  DevBuf<int32_t> flags;          // [4]: 0 any active, 1 any reorth
  DevBuf<double> est;             // [nrhs] residual estimate / ||b||
  int32_t* h_flags = nullptr;     // pinned
  double* h_small = nullptr;      // pinned [3 * nrhs]
  int nblk = 0;
  ~Workspace() {
    if (h_flags) cudaFreeHost(h_flags);
    if (h_small) cudaFreeHost(h_small);
  }
};

void free_workspace(Problem& P) {
  delete P.ws;
  P.ws = nullptr;
}

static Workspace& workspace(Problem& P, int nrhs, int m) {
  const int64_t n = P.fine.n_dof;
  const size_t zsz = P.precision == MX_MIXED ? sizeof(float2) : sizeof(double2);
  Workspace* W = P.ws;
  if (W && W->nrhs == nrhs && W->m >= m && W->n == n) return *W;
  delete W;
  W = P.ws = new Workspace();
  W->nrhs = nrhs;
  W->m = m;
  W->n = n;
  W->zsz = zsz;
  const int64_t nv = n * nrhs;
  W->V.alloc((size_t)(m + 1) * nv);
  W->Z.alloc((size_t)m * nv * zsz);
  W->w.alloc(nv);
  W->b.alloc(nv);
  W->x.alloc(nv);
  W->r.alloc(nv);
  if (P.precision == MX_MIXED) {
    W->hs.alloc((size_t)(m + 2) * nrhs);
    W->g2.alloc((size_t)(m + 1) * nrhs);
    W->inv2.alloc(nrhs);
  }
  W->loc.alloc((size_t)P.sum_local * nrhs * zsz);
  if (P.coarse_m) W->yc.alloc((size_t)P.n_c * nrhs);
  W->H.alloc((size_t)m * (m + 1) * nrhs);
  W->cs.alloc((size_t)m * nrhs);
  W->sn.alloc((size_t)m * nrhs);
  W->g.alloc((size_t)(m + 1) * nrhs);
  W->y.alloc((size_t)m * nrhs);
  W->nblk = 4 * sm_count();
  W->hpart.alloc((size_t)W->nblk * (m + 2) * nrhs);
  W->h2.alloc((size_t)(m + 2) * nrhs);
  W->h1.alloc((size_t)(m + 2) * nrhs);
  W->npart.alloc((size_t)W->nblk * nrhs);
  W->bnorm.alloc(nrhs);
  W->wnorm0.alloc(nrhs);
  W->active.alloc(nrhs);
  W->flags.alloc(4);
  W->est.alloc(nrhs);
  MX_CUDA(cudaHostAlloc(&W->h_flags, 16, cudaHostAllocDefault));
  MX_CUDA(cudaHostAlloc(&W->h_small, sizeof(double) * 3 * nrhs, cudaHostAllocDefault));
  return *W;
}

// z = sum of the local solutions held in W.loc (all of them, or the owner's only when `own`
// is given) + (R^0)^T y0 when `coarse` (y0 in W.yc); z in ztype, zc the promoted copy.
static void scatter(Problem& P, Workspace& W, void* z, int ztype, int nrhs, bool local, bool coarse,
                    const int32_t* own, double2* zc) {
  cudaStream_t s = P.stream;
  const bool mixed = P.precision == MX_MIXED;
  const int64_t work = P.fine.n_dof * nrhs;
  const int32_t* tp = coarse ? P.R0T.rowptr.p : nullptr;
  const unsigned grid = grid_for(work, 256, 152LL * 32);
  const double lsz = mixed ? 8.0 : 16.0, zb = ztype == 0 ? 16.0 : 8.0;
  ProfScope ps(K_SCATTER, s, 1,
               (local ? (lsz * nrhs + 4.0) * (double)P.sum_local : 0.0) + 4.0 * (P.fine.n_dof + 1) +
                   (coarse ? 12.0 * P.R0T.nnz + 4.0 * P.fine.n_dof + lsz * (double)P.n_c * nrhs : 0.0) +
                   zb * (double)work,
               (local ? 2.0 * (double)P.sum_local * nrhs : 0.0) + (coarse ? 4.0 * (double)P.R0T.nnz * nrhs : 0.0));
#define MX_SCATTER(LT, CT, ZT, AT, TV)                                                                        \
  MX_LAUNCH(k_scatter<LT, CT, ZT, AT><<<grid, 256, 0, s>>>(P.fine.n_dof, nrhs, P.inv_ptr.p, P.inv_pos.p, own,       \
                                                           (const LT*)W.loc.p, tp, P.R0T.col.p, TV,              \
                                                           (const CT*)W.yc.p, local ? 1 : 0, (ZT*)z, zc))
  if (mixed) {
    if (coarse && P.R0T_valf.n != (size_t)P.R0T.nnz) {
      P.R0T_valf.alloc(P.R0T.nnz);
      MX_LAUNCH(k_to_f32<<<grid_for(P.R0T.nnz, 256), 256, 0, s>>>(P.R0T.nnz, P.R0T.val.p, P.R0T_valf.p));
      MX_CHECK_LAUNCH();
    }
    if (nrhs % 2 == 0) {
      const unsigned grid2 = grid_for(P.fine.n_dof * (nrhs / 2), 256, 152LL * 32);
      const float4* l4 = reinterpret_cast<const float4*>(W.loc.p);
      const float4* y4 = reinterpret_cast<const float4*>(W.yc.p);
      if (ztype == 0)
        MX_LAUNCH(k_scatter2<double2><<<grid2, 256, 0, s>>>(P.fine.n_dof, nrhs, P.inv_ptr.p, P.inv_pos.p, own, l4, tp,
                                                            P.R0T.col.p, P.R0T_valf.p, y4, local ? 1 : 0,
                                                            (double2*)z, zc));
      else
        MX_LAUNCH(k_scatter2<float2><<<grid2, 256, 0, s>>>(P.fine.n_dof, nrhs, P.inv_ptr.p, P.inv_pos.p, own, l4, tp,
                                                           P.R0T.col.p, P.R0T_valf.p, y4, local ? 1 : 0,
                                                           (float2*)z, zc));
    } else if (ztype == 0) {
      MX_SCATTER(float2, float2, double2, float, P.R0T_valf.p);
    } else {
      MX_SCATTER(float2, float2, float2, float, P.R0T_valf.p);
    }
  } else {
    if (ztype == 0) MX_SCATTER(double2, double2, double2, double, P.R0T.val.p);
    else MX_SCATTER(double2, double2, float2, double, P.R0T.val.p);
  }
#undef MX_SCATTER
  MX_CHECK_LAUNCH();
}

// t = v - t (v c128 or complex double-float)
__global__ void k_sub_from(int64_t nv, const void* v, int vtype, double2* t) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    double2 a;
    if (vtype == 3) {
      const float4 d = reinterpret_cast<const float4*>(v)[i];
      a = make_double2((double)d.x + (double)d.z, (double)d.y + (double)d.w);
    } else if (vtype == 1) {
      const float2 d = reinterpret_cast<const float2*>(v)[i];
      a = make_double2(d.x, d.y);
    } else {
      a = reinterpret_cast<const double2*>(v)[i];
    }
    t[i] = make_double2(a.x - t[i].x, a.y - t[i].y);
  }
}

// z = u + g in ztype; zc the promoted copy of the stored z
template <typename ZT, typename UT>
__global__ void k_add_out(int64_t nv, const UT* u, const UT* g, ZT* z, double2* zc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = to_c128(u[i]), b = to_c128(g[i]);
    const ZT zv = conv<ZT>(make_double2(a.x + b.x, a.y + b.y));
    z[i] = zv;
    if (zc) zc[i] = to_c128(zv);
  }
}

void precond_apply(Problem& P, const void* v, void* z, int ztype, int nrhs, int levels, double2* zc, int vtype) {
  Workspace& W = workspace(P, nrhs, P.ws ? std::max(P.ws->m, 1) : 1);
  cudaStream_t s = P.stream;
  const int kind = P.prec_kind;
  const int32_t* own = nullptr;
  if (kind != MX_PREC_AS) {
    build_owner(P);
    own = P.own_pos.p;
  }
  if ((kind == MX_PREC_HRAS || kind == MX_PREC_ADEF1) && P.coarse_m) {
    // two-level hybrid forms (Sec. 6.3): G v, t = v - A G v, u = B_RAS1^{-1} t, then
    // ADEF1: z = u + G v;  HRAS: z = u + G (v - A u)  (= (I - G A) u + G v)
    // mixed form: G v and u are c64 (their parts are), so the products with A_{xi_prec}
    // run on the double-float operator; FP64 form: c128 and the FP64 operator
    const bool mixed = P.precision == MX_MIXED;
    const int64_t nv = P.fine.n_dof * nrhs;
    W.pv.ensure((size_t)3 * nv);
    double2* gv = W.pv.p;
    double2* t = W.pv.p + nv;
    double2* u = W.pv.p + 2 * nv;
    const int ut = mixed ? 1 : 0;  // storage type of gv and u
    auto apply_a = [&](const double2* x, double2* y) {
      if (mixed) spmv_df_c128(P, P.xi_prec, reinterpret_cast<const float2*>(x), y, nrhs, s);
      else spmv(P, P.xi_prec, x, 0, y, nrhs, s);
    };
    const unsigned gv_grid = grid_for(nv, 256);
    coarse_solve(P, v, vtype, W.yc.p, nrhs);
    scatter(P, W, gv, ut, nrhs, false, true, nullptr, nullptr);
    apply_a(gv, t);
    MX_LAUNCH(k_sub_from<<<gv_grid, 256, 0, s>>>(nv, v, vtype, t));
    MX_CHECK_LAUNCH();
    local_solves(P, t, 0, W.loc.p, nrhs);
    scatter(P, W, u, ut, nrhs, true, false, own, nullptr);
    if (kind == MX_PREC_HRAS) {
      apply_a(u, t);
      MX_LAUNCH(k_sub_from<<<gv_grid, 256, 0, s>>>(nv, v, vtype, t));
      MX_CHECK_LAUNCH();
      coarse_solve(P, t, 0, W.yc.p, nrhs);
      scatter(P, W, gv, ut, nrhs, false, true, nullptr, nullptr);
    }
    if (mixed) {
      const float2* uf = reinterpret_cast<const float2*>(u);
      const float2* gf = reinterpret_cast<const float2*>(gv);
      if (ztype == 0) MX_LAUNCH(k_add_out<double2, float2><<<gv_grid, 256, 0, s>>>(nv, uf, gf, (double2*)z, zc));
      else MX_LAUNCH(k_add_out<float2, float2><<<gv_grid, 256, 0, s>>>(nv, uf, gf, (float2*)z, zc));
    } else {
      if (ztype == 0) MX_LAUNCH(k_add_out<double2, double2><<<gv_grid, 256, 0, s>>>(nv, u, gv, (double2*)z, zc));
      else MX_LAUNCH(k_add_out<float2, double2><<<gv_grid, 256, 0, s>>>(nv, u, gv, (float2*)z, zc));
    }
    MX_CHECK_LAUNCH();
    return;
  }
  // (running the coarse solve concurrently with the local solves gains under 1 % of the step:
  // both read HBM, and the memory-bound local solves lose what the coarse solve saves)
  if (levels & 1) local_solves(P, v, vtype, W.loc.p, nrhs);
  const bool coarse = (levels & 2) && P.coarse_m;
  if (coarse) coarse_solve(P, v, vtype, W.yc.p, nrhs);
  scatter(P, W, z, ztype, nrhs, (levels & 1) != 0, coarse, own, zc);
}

// ---- Arnoldi kernels ----------------------------------------------------------------
// Partial dots: block `blk` owns rows [x0, x1). Warp w handles basis indices i = w, w+8,
// ...; lanes are (xl, r) with r fastest (RP = nrhs rounded up to a power of two <= 32,
// XL = 32 / RP rows per warp step). Index i == nvec - 1 + extra uses w itself (its norm).
// hpart[blk][i][r] = sum_{x in block} conj(V_i[x][r]) w[x][r]
template <int RP>
__global__ void __launch_bounds__(256) k_dots(int64_t n, int nrhs, int nvec, int with_norm, const double2* __restrict__ V,
                                              const double2* __restrict__ w, const int32_t* __restrict__ active,
                                              double2* __restrict__ hpart, const double2* __restrict__ extra = nullptr) {
  constexpr int XL = 32 / RP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane % RP, xl = lane / RP;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
  const int total = nvec + with_norm;
  const int64_t nv = n * nrhs;
  const bool on = r < nrhs && active[min(r, nrhs - 1)];
  for (int i = warp; i < total; i += 8) {
    const double2* Vi = (i < nvec) ? V + (int64_t)i * nv : (extra ? extra : w);
    double ax = 0, ay = 0;
    if (on)
      for (int64_t x = x0 + xl; x < x1; x += XL) {
        const double2 a = Vi[x * nrhs + r];
        const double2 c = w[x * nrhs + r];
        ax = fma(a.x, c.x, ax);
        ax = fma(a.y, c.y, ax);
        ay = fma(a.x, c.y, ay);
        ay = fma(-a.y, c.x, ay);
      }
#pragma unroll
    for (int o = RP; o < 32; o <<= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (xl == 0 && r < nrhs) hpart[((int64_t)blockIdx.x * (total) + i) * nrhs + r] = make_double2(ax, ay);
  }
}

// h[i][r] = sum_blk hpart[blk][i][r]: one warp per output, lane l sums blocks l, l + 32, ...,
// then a fixed shuffle tree (deterministic)
__global__ void k_reduce_dots(int nblk, int total, int nrhs, const double2* hpart, double2* h) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total * nrhs; t += warps) {
    double ax = 0, ay = 0;
    for (int b = lane; b < nblk; b += 32) {
      const double2 v = hpart[(int64_t)b * total * nrhs + t];
      ax += v.x;
      ay += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) h[t] = make_double2(ax, ay);
  }
}

// w[x][r] -= sum_{i < nvec} V_i[x][r] h[i][r]; npart[blk][r] = sum over the block of |w|^2
template <int RP>
__global__ void __launch_bounds__(256) k_orth_update(int64_t n, int nrhs, int nvec, const double2* __restrict__ V,
                                                     const double2* __restrict__ h, const int32_t* __restrict__ active,
                                                     double2* __restrict__ w, double* __restrict__ npart) {
  constexpr int XL = 32 / RP;
  __shared__ double sh[8][RP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane % RP, xl = lane / RP;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
  const int64_t nv = n * nrhs;
  const bool on = r < nrhs && active[min(r, nrhs - 1)];
  double nrm = 0;
  if (on)
    for (int64_t x = x0 + warp * XL + xl; x < x1; x += 8 * XL) {
      double2 acc = w[x * nrhs + r];
      for (int i = 0; i < nvec; ++i) {
        const double2 a = V[(int64_t)i * nv + x * nrhs + r];
        const double2 c = h[i * nrhs + r];
        acc.x = fma(-a.x, c.x, acc.x);
        acc.x = fma(a.y, c.y, acc.x);
        acc.y = fma(-a.x, c.y, acc.y);
        acc.y = fma(-a.y, c.x, acc.y);
      }
      w[x * nrhs + r] = acc;
      nrm = fma(acc.x, acc.x, nrm);
      nrm = fma(acc.y, acc.y, nrm);
    }
#pragma unroll
  for (int o = RP; o < 32; o <<= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (xl == 0) sh[warp][r] = nrm;
  __syncthreads();
  if (threadIdx.x < RP && threadIdx.x < nrhs) {
    double s = 0;
    for (int wq = 0; wq < 8; ++wq) s += sh[wq][threadIdx.x];
    npart[(int64_t)blockIdx.x * nrhs + threadIdx.x] = s;
  }
}

// After pass p: store h (accumulated over passes) into column j of H, the new norm,
// and decide whether a second pass is needed (DGKS, eta = 1/sqrt(2)).
__global__ void k_arnoldi_finish(int nblk, int nrhs, int j, int m, int pass, const double2* h2, const double* npart,
                                 double2* H, double* wnorm0, int32_t* active, int32_t* flags) {
  const int r = threadIdx.x;
  if (r == 0 && pass == 0) flags[1] = 0;
  __syncthreads();
  if (r >= nrhs) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += npart[(int64_t)b * nrhs + r];
  const double nw = sqrt(s);
  if (!active[r]) return;
  double2* Hc = H + (int64_t)j * (m + 1) * nrhs;
  for (int i = 0; i <= j; ++i) {
    const double2 v = h2[i * nrhs + r];
    if (pass == 0) Hc[i * nrhs + r] = v;
    else Hc[i * nrhs + r] = make_double2(Hc[i * nrhs + r].x + v.x, Hc[i * nrhs + r].y + v.y);
  }
  if (pass == 0) wnorm0[r] = sqrt(h2[(j + 1) * nrhs + r].x);  // ||w|| before orthogonalisation
  Hc[(j + 1) * nrhs + r] = make_double2(nw, 0.0);
  if (pass == 0 && nw < 0.7071067811865476 * wnorm0[r]) atomicOr(&flags[1], 1);
}

// Weighted Arnoldi (D-inner product), per right-hand side. stage 0, after the inner products
// of w (h1, entry j+1 = ||w||_D^2) and of the updated w' (h2, entry j+1 = ||w'||_D^2): store
// column j, its subdiagonal ||w'||_D and the DGKS decision. stage 1, after the second update
// with h2: add h2 to the column and take the norm by Pythagoras, ||w''||^2 = ||w'||^2 - |h2|^2
// (the correction is small when it is needed).
__global__ void k_arnoldi_finish_w(int nrhs, int j, int m, int stage, const double2* h1, const double2* h2, double2* H,
                                   const int32_t* active, int32_t* flags) {
  const int r = threadIdx.x;
  if (r == 0 && stage == 0) flags[1] = 0;
  __syncthreads();
  if (r >= nrhs || !active[r]) return;
  double2* Hc = H + (int64_t)j * (m + 1) * nrhs;
  const double n1 = sqrt(fmax(h2[(j + 1) * nrhs + r].x, 0.0));
  if (stage == 0) {
    for (int i = 0; i <= j; ++i) Hc[i * nrhs + r] = h1[i * nrhs + r];
    const double n0 = sqrt(fmax(h1[(j + 1) * nrhs + r].x, 0.0));
    Hc[(j + 1) * nrhs + r] = make_double2(n1, 0.0);
    if (n1 < 0.7071067811865476 * n0) atomicOr(&flags[1], 1);
  } else {
    double c = 0;
    for (int i = 0; i <= j; ++i) {
      const double2 v = h2[i * nrhs + r];
      Hc[i * nrhs + r] = make_double2(Hc[i * nrhs + r].x + v.x, Hc[i * nrhs + r].y + v.y);
      c += v.x * v.x + v.y * v.y;
    }
    Hc[(j + 1) * nrhs + r] = make_double2(sqrt(fmax(n1 * n1 - c, 0.0)), 0.0);
  }
}

// Two-pass classical Gram-Schmidt of the mixed form, per right-hand side. stage 0, after the
// pass-1 inner products h (c64 accuracy): column j of H = h. stage 1, after the double-float
// update (npart: ||w'||^2 partials) and the pass-2 inner products h: add h to the column,
// ||w''||^2 = ||w'||^2 - |h|^2 (Pythagoras; the correction is small) into the subdiagonal,
// g = h rounded to c64 and inv = 1 / ||w''|| as a double-float (0 for a zero norm or a
// finished right-hand side) for the fused correction and normalisation.
__global__ void k_cgs2_finish(int nblk, int nrhs, int j, int m, int stage, const double2* h, const double* npart,
                              double2* H, const int32_t* active, float2* g, float2* inv) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  if (!active[r]) {
    if (stage == 1) {
      for (int i = 0; i <= j; ++i) g[i * nrhs + r] = make_float2(0.f, 0.f);
      inv[r] = make_float2(0.f, 0.f);
    }
    return;
  }
  double2* Hc = H + (int64_t)j * (m + 1) * nrhs;
  if (stage == 0) {
    for (int i = 0; i <= j; ++i) Hc[i * nrhs + r] = h[i * nrhs + r];
    return;
  }
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += npart[(int64_t)b * nrhs + r];
  double c = 0;
  for (int i = 0; i <= j; ++i) {
    const double2 v = h[i * nrhs + r];
    Hc[i * nrhs + r] = make_double2(Hc[i * nrhs + r].x + v.x, Hc[i * nrhs + r].y + v.y);
    c += v.x * v.x + v.y * v.y;
    g[i * nrhs + r] = make_float2((float)v.x, (float)v.y);
  }
  const double nw = sqrt(fmax(s - c, 0.0));
  Hc[(j + 1) * nrhs + r] = make_double2(nw, 0.0);
  const double iv = nw > 0 ? 1.0 / nw : 0.0;
  const float hi = (float)iv;
  inv[r] = make_float2(hi, (float)(iv - (double)hi));
}

// npart[blk][q] = partial sums of Re(conj(r) y) (y = D r): the D-norm of r squared
__global__ void k_wnorm_partials(int64_t n, int nrhs, const double2* r, const double2* y, double* npart) {
  __shared__ double sh[256];
  const int64_t nv = n * nrhs;
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x) * nrhs;
  const int64_t t0 = blockIdx.x * chunk, t1 = min(nv, t0 + chunk);
  double acc = 0;
  const int q = threadIdx.x % nrhs;
  const int lanes = 256 / nrhs;
  const int li = threadIdx.x / nrhs;
  if (li < lanes)
    for (int64_t t = t0 + (int64_t)li * nrhs + q; t < t1; t += (int64_t)lanes * nrhs) {
      acc = fma(r[t].x, y[t].x, acc);
      acc = fma(r[t].y, y[t].y, acc);
    }
  sh[threadIdx.x] = (li < lanes) ? acc : 0.0;
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double s = 0;
    for (int l = 0; l < lanes; ++l) s += sh[l * nrhs + threadIdx.x];
    npart[(int64_t)blockIdx.x * nrhs + threadIdx.x] = s;
  }
}

// v_{j+1} = w / h_{j+1,j}
__global__ void k_normalize(int64_t nv, int nrhs, int j, int m, const double2* H, const int32_t* active,
                            const double2* w, double2* vnext) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const double hn = H[((int64_t)j * (m + 1) + j + 1) * nrhs + r].x;
    const double inv = (hn > 0 && active[r]) ? 1.0 / hn : 0.0;
    vnext[t] = make_double2(w[t].x * inv, w[t].y * inv);
  }
}

// Givens update of column j for every active right-hand side (one thread each).
__global__ void k_givens(int nrhs, int j, int m, double tol, const double* bnorm, double2* H, double* cs,
                         double2* sn, double2* g, int32_t* active, double* est, int32_t* flags) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs || !active[r]) return;
  double2* Hc = H + (int64_t)j * (m + 1) * nrhs;
  for (int i = 0; i < j; ++i) {
    const double c = cs[i * nrhs + r];
    const double2 s = sn[i * nrhs + r];
    const double2 a = Hc[i * nrhs + r], b = Hc[(i + 1) * nrhs + r];
    // [c s; -conj(s) c] [a; b]
    Hc[i * nrhs + r] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
    Hc[(i + 1) * nrhs + r] = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
  }
  const double2 a = Hc[j * nrhs + r], b = Hc[(j + 1) * nrhs + r];
  const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
  double c;
  double2 s;
  if (bb == 0) { c = 1; s = make_double2(0, 0); }
  else if (aa == 0) { c = 0; s = make_double2(b.x / bb, -b.y / bb); }
  else {
    const double t = hypot(aa, bb);
    c = aa / t;
    const double2 ph = make_double2(a.x / aa, a.y / aa);  // a / |a|
    // s = (a/|a|) conj(b) / t
    s = make_double2((ph.x * b.x + ph.y * b.y) / t, (ph.y * b.x - ph.x * b.y) / t);
  }
  cs[j * nrhs + r] = c;
  sn[j * nrhs + r] = s;
  Hc[j * nrhs + r] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
  Hc[(j + 1) * nrhs + r] = make_double2(0, 0);
  const double2 gj = g[j * nrhs + r];
  // g_{j+1} = -conj(s) g_j ; g_j = c g_j
  g[(j + 1) * nrhs + r] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  g[j * nrhs + r] = make_double2(c * gj.x, c * gj.y);
  const double2 gn = g[(j + 1) * nrhs + r];
  est[r] = hypot(gn.x, gn.y) / bnorm[r];
}

// y = R^{-1} g for the first k columns (R upper triangular in H after the rotations).
__global__ void k_backsolve(int nrhs, int m, const int32_t* kcols, const double2* H, const double2* g, double2* y) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int k = kcols[r];
  for (int i = k - 1; i >= 0; --i) {
    double2 s = g[i * nrhs + r];
    for (int c = i + 1; c < k; ++c) {
      const double2 h = H[((int64_t)c * (m + 1) + i) * nrhs + r];
      const double2 yc = y[c * nrhs + r];
      s.x -= h.x * yc.x - h.y * yc.y;
      s.y -= h.x * yc.y + h.y * yc.x;
    }
    const double2 d = H[((int64_t)i * (m + 1) + i) * nrhs + r];
    const double dd = d.x * d.x + d.y * d.y;
    y[i * nrhs + r] = make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd);
  }
}

// x[x][r] += sum_{i < k_r} Z_i[x][r] y_i[r]
template <typename ZT>
__global__ void k_update_x(int64_t n, int nrhs, const int32_t* kcols, const ZT* Z, const double2* y, double2* x) {
  const int64_t nv = n * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const int k = kcols[r];
    double2 acc = x[t];
    for (int i = 0; i < k; ++i) {
      const double2 z = to_c128(Z[(int64_t)i * nv + t]);
      const double2 c = y[i * nrhs + r];
      acc.x = fma(z.x, c.x, acc.x);
      acc.x = fma(-z.y, c.y, acc.x);
      acc.y = fma(z.x, c.y, acc.y);
      acc.y = fma(z.y, c.x, acc.y);
    }
    x[t] = acc;
  }
}

// r = b - A x (A x already in r); npart[blk][r] = partial |r|^2
__global__ void k_residual(int64_t n, int nrhs, const double2* b, double2* r, double* npart) {
  __shared__ double sh[256];
  const int64_t nv = n * nrhs;
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x) * nrhs;
  const int64_t t0 = blockIdx.x * chunk, t1 = min(nv, t0 + chunk);
  // thread owns right-hand side q = threadIdx.x % nrhs when nrhs divides 256
  double acc = 0;
  const int q = threadIdx.x % nrhs;
  const int lanes = 256 / nrhs;
  const int li = threadIdx.x / nrhs;
  if (li < lanes)
    for (int64_t t = t0 + (int64_t)li * nrhs + q; t < t1; t += (int64_t)lanes * nrhs) {
      const double2 v = make_double2(b[t].x - r[t].x, b[t].y - r[t].y);
      r[t] = v;
      acc = fma(v.x, v.x, acc);
      acc = fma(v.y, v.y, acc);
    }
  sh[threadIdx.x] = (li < lanes) ? acc : 0.0;
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double s = 0;
    for (int l = 0; l < lanes; ++l) s += sh[l * nrhs + threadIdx.x];
    npart[(int64_t)blockIdx.x * nrhs + threadIdx.x] = s;
  }
}

// norms from partials; restart set-up: v0 = r / beta, g = (beta, 0, ...)
__global__ void k_restart(int nblk, int nrhs, int m, const double* npart, const double* bnorm, double tol,
                          int32_t* active, double* beta_out, double2* g) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += npart[(int64_t)b * nrhs + r];
  const double beta = sqrt(s);
  beta_out[r] = beta;
  for (int i = 0; i <= m; ++i) g[i * nrhs + r] = make_double2(0, 0);
  g[r] = make_double2(beta, 0);
  active[r] = (beta > tol * bnorm[r]) ? 1 : 0;
}

__global__ void k_scale_v0(int64_t nv, int nrhs, const double* beta, const int32_t* active, const double2* r, double2* v0) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % nrhs);
    const double inv = (active[q] && beta[q] > 0) ? 1.0 / beta[q] : 0.0;
    v0[t] = make_double2(r[t].x * inv, r[t].y * inv);
  }
}

__global__ void k_copy_norm(int nrhs, const double* beta, double* bnorm) {
  const int r = threadIdx.x;
  if (r < nrhs) bnorm[r] = beta[r];
}

template <int RP>
static void launch_dots(Workspace& W, int64_t n, int nvec, int with_norm, const double2* V, cudaStream_t s,
                        const double2* target, const double2* extra) {
  MX_LAUNCH(k_dots<RP><<<W.nblk, 256, 0, s>>>(n, W.nrhs, nvec, with_norm, V, target, W.active.p, W.hpart.p, extra));
}
template <int RP>
static void launch_update(Workspace& W, int64_t n, int nvec, cudaStream_t s) {
  MX_LAUNCH(k_orth_update<RP><<<W.nblk, 256, 0, s>>>(n, W.nrhs, nvec, W.V.p, W.h2.p, W.active.p, W.w.p, W.npart.p));
}

// h = V^H target (+ extra^H target, or |target|^2 when extra is null, as entry nvec when
// with_norm); target defaults to w
static void dots(Workspace& W, int64_t n, int nvec, int with_norm, cudaStream_t s, const double2* target = nullptr,
                 const double2* extra = nullptr) {
  const int nr = W.nrhs;
  if (!target) target = W.w.p;
  {
    // V_0..V_{nvec-1} and w read once each
    ProfScope ps(K_DOTS, s, 1, 16.0 * (nvec + 1) * (double)n * nr, 8.0 * (nvec + with_norm) * (double)n * nr);
    if (nr <= 1) launch_dots<1>(W, n, nvec, with_norm, W.V.p, s, target, extra);
    else if (nr <= 2) launch_dots<2>(W, n, nvec, with_norm, W.V.p, s, target, extra);
    else if (nr <= 4) launch_dots<4>(W, n, nvec, with_norm, W.V.p, s, target, extra);
    else if (nr <= 8) launch_dots<8>(W, n, nvec, with_norm, W.V.p, s, target, extra);
    else if (nr <= 16) launch_dots<16>(W, n, nvec, with_norm, W.V.p, s, target, extra);
    else launch_dots<32>(W, n, nvec, with_norm, W.V.p, s, target, extra);
    MX_CHECK_LAUNCH();
  }
  const int total = nvec + with_norm;
  ProfScope ps(K_ARNOLDI_SMALL, s);
  MX_LAUNCH(k_reduce_dots<<<grid_for((int64_t)total * nr * 32, 256), 256, 0, s>>>(W.nblk, total, nr, W.hpart.p, W.h2.p));
  MX_CHECK_LAUNCH();
}

// planes of the mixed-form basis inside W.V: all c64 roundings first, then all remainders
static float2* basis_hi(Workspace& W) { return reinterpret_cast<float2*>(W.V.p); }
static float2* basis_lo(Workspace& W) { return reinterpret_cast<float2*>(W.V.p) + (int64_t)(W.m + 1) * W.n * W.nrhs; }

// mixed form: double-float passes over the basis, FP64 reduction of the block partials
static void dots_mixed(Workspace& W, int64_t n, int nvec, int with_norm, cudaStream_t s, int32_t* timeout,
                       const double2* target = nullptr, const double2* extra = nullptr) {
  // one resident wave: the lane-parallel kernels hold 64 KB of accumulators per block (3 per
  // SM), the staged one 108 KB of stages (2 per SM)
  const int nb = dots_df(std::min(W.nblk, 3 * sm_count()), n, W.nrhs, nvec, with_norm, basis_hi(W), basis_lo(W),
                         reinterpret_cast<const float4*>(target ? target : W.w.p), W.active.p, W.hpart.p, s,
                         reinterpret_cast<const float4*>(extra), timeout);
  const int total = nvec + with_norm;
  ProfScope ps(K_ARNOLDI_SMALL, s);
  MX_LAUNCH(k_reduce_dots<<<grid_for((int64_t)total * W.nrhs * 32, 256), 256, 0, s>>>(nb, total, W.nrhs, W.hpart.p,
                                                                                   W.h2.p));
  MX_CHECK_LAUNCH();
}

static void orth_update(Workspace& W, int64_t n, int nvec, cudaStream_t s) {
  const int nr = W.nrhs;
  // V_0..V_{nvec-1} read once, w read and written once
  ProfScope ps(K_ORTH_UPDATE, s, 1, 16.0 * (nvec + 2) * (double)n * nr, 8.0 * (nvec + 0.25) * (double)n * nr);
  if (nr <= 1) launch_update<1>(W, n, nvec, s);
  else if (nr <= 2) launch_update<2>(W, n, nvec, s);
  else if (nr <= 4) launch_update<4>(W, n, nvec, s);
  else if (nr <= 8) launch_update<8>(W, n, nvec, s);
  else if (nr <= 16) launch_update<16>(W, n, nvec, s);
  else launch_update<32>(W, n, nvec, s);
  MX_CHECK_LAUNCH();
}

// weighted GMRES: replace the Euclidean partials of r in npart by those of ||r||_D^2
// (D r formed in W.w, which is free at restarts)
static void weighted_norm_partials(Problem& P, Workspace& W, cudaStream_t s) {
  spmv_km(P, -P.k * P.k, 0.0, W.r.p, 0, W.w.p, W.nrhs, s);
  ProfScope ps(K_RESIDUAL, s);
  MX_LAUNCH(k_wnorm_partials<<<W.nblk, 256, 0, s>>>(W.n, W.nrhs, W.r.p, W.w.p, W.npart.p));
  MX_CHECK_LAUNCH();
}

static void true_residual(Problem& P, Workspace& W, cudaStream_t s) {
  spmv(P, P.xi_prob, W.x.p, 0, W.r.p, W.nrhs, s);
  {
    ProfScope ps(K_RESIDUAL, s, 1, 48.0 * (double)W.n * W.nrhs, 6.0 * (double)W.n * W.nrhs);
    MX_LAUNCH(k_residual<<<W.nblk, 256, 0, s>>>(W.n, W.nrhs, W.b.p, W.r.p, W.npart.p));
    MX_CHECK_LAUNCH();
  }
  if (P.weighted) weighted_norm_partials(P, W, s);
}

__global__ void k_fill_i32(int n, int32_t v, int32_t* p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

void fill_i32(int32_t* p, int n, int32_t v, cudaStream_t s) {
  MX_LAUNCH(k_fill_i32<<<1, 256, 0, s>>>(n, v, p));
  MX_CHECK_LAUNCH();
}

void batched_dots(const double2* V, const double2* w, int64_t n, int nrhs, int nvec, double2* h, double2* partials,
                  int nblk, const int32_t* ones, cudaStream_t s) {
  MX_REQUIRE(nrhs >= 1 && nrhs <= 32 && nvec >= 1 && n >= 1 && nblk >= 1, MX_EINVAL, "bad batched_dots sizes");
#define MX_DOTS(RP) MX_LAUNCH(k_dots<RP><<<nblk, 256, 0, s>>>(n, nrhs, nvec, 0, V, w, ones, partials))
  if (nrhs <= 1) MX_DOTS(1);
  else if (nrhs <= 2) MX_DOTS(2);
  else if (nrhs <= 4) MX_DOTS(4);
  else if (nrhs <= 8) MX_DOTS(8);
  else if (nrhs <= 16) MX_DOTS(16);
  else MX_DOTS(32);
#undef MX_DOTS
  MX_CHECK_LAUNCH();
  MX_LAUNCH(k_reduce_dots<<<grid_for((int64_t)nvec * nrhs * 32, 256), 256, 0, s>>>(nblk, nvec, nrhs, partials, h));
  MX_CHECK_LAUNCH();
}

__global__ void k_zero_cols(int64_t nv, int nrhs, const int32_t* mask, double2* x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x)
    if (mask[t % nrhs]) x[t] = make_double2(0, 0);
}

int gmres_solve(Problem& P, const double2* b, double2* x, int nrhs, double tol, int restart, int max_it,
                mx_rhs_stats* stats, SlotHook* hook) {
  MX_REQUIRE(P.factored, MX_ENOTFACTORED, "mx_solve before mx_factor");
  MX_REQUIRE(nrhs >= 1 && nrhs <= 32, MX_EINVAL, "nrhs must be in 1..32 per batch");
  MX_REQUIRE(max_it >= 1, MX_EINVAL, "max_it must be >= 1");
  cudaStream_t s = P.stream;
  // status[2] counts bounded tensor-core waits that ran out; the local solves of this
  // solve report into it, read back with the solution below
  MX_CUDA(cudaMemsetAsync(P.status.p + 2, 0, sizeof(int32_t), s));
  const int m = restart > 0 ? std::min(restart, max_it) : max_it;
  Workspace& W = workspace(P, nrhs, m);
  const int64_t n = P.fine.n_dof, nv = n * nrhs;
  const bool mixed = P.precision == MX_MIXED;
  const int ztype = mixed ? 1 : 0;
  const size_t zsz = W.zsz;
  int64_t launches = 0;
  std::vector<int32_t> its(nrhs, 0), done(nrhs, 0), kcols(nrhs, 0), reported(nrhs, 0);
  std::vector<double> rel(nrhs, 1.0), estv(nrhs, 1.0), bn(nrhs, 0.0);
  DevBuf<int32_t> dk(nrhs);
  DevBuf<double> beta(nrhs);

  MX_CUDA(cudaMemcpyAsync(W.b.p, b, nv * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  MX_CUDA(cudaMemsetAsync(W.x.p, 0, nv * sizeof(double2), s));
  // ||b||: residual of x = 0
  MX_CUDA(cudaMemsetAsync(W.r.p, 0, nv * sizeof(double2), s));
  MX_LAUNCH(k_residual<<<W.nblk, 256, 0, s>>>(n, nrhs, W.b.p, W.r.p, W.npart.p));
  if (P.weighted) weighted_norm_partials(P, W, s);  // ||b||_D
  MX_CUDA(cudaMemsetAsync(W.active.p, 0, nrhs * 4, s));
  MX_LAUNCH(k_restart<<<1, 32, 0, s>>>(W.nblk, nrhs, m, W.npart.p, W.bnorm.p, -1.0, W.active.p, beta.p, W.g.p));
  MX_LAUNCH(k_copy_norm<<<1, 32, 0, s>>>(nrhs, beta.p, W.bnorm.p));
  launches += 3;
  MX_CHECK_LAUNCH();
  MX_CUDA(cudaMemcpyAsync(bn.data(), W.bnorm.p, nrhs * 8, cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  // zero right-hand sides converge at once with x = 0
  std::vector<int32_t> act(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    act[r] = bn[r] > 0;
    if (!act[r]) { done[r] = 1; rel[r] = 0; estv[r] = 0; }
  }
  MX_CUDA(cudaMemcpyAsync(W.active.p, act.data(), nrhs * 4, cudaMemcpyHostToDevice, s));
  if (mixed) {
    scale_v0_df(nv, nrhs, beta.p, W.active.p, W.r.p, basis_hi(W), basis_lo(W), s);
  } else {
    MX_LAUNCH(k_scale_v0<<<grid_for(nv, 256), 256, 0, s>>>(nv, nrhs, beta.p, W.active.p, W.r.p, W.V.p));
    MX_CHECK_LAUNCH();
  }
  ++launches;

  int total_its = 0, restarts = 0;
  const unsigned gv = grid_for(nv, 256);
  while (std::any_of(act.begin(), act.end(), [](int32_t a) { return a != 0; })) {
    std::vector<int32_t> start_active = act;
    for (int j = 0; j < m; ++j) {
      unsigned char* zj = W.Z.p + (size_t)j * nv * zsz;
      // z_j = B^{-1} v_j ; w = A z_j (mixed: the preconditioner reads the c64 plane of v_j,
      // w is a double-float, z_j is c64)
      if (mixed) precond_apply(P, basis_hi(W) + (int64_t)j * nv, zj, ztype, nrhs, 3, nullptr, 1);
      else precond_apply(P, W.V.p + (int64_t)j * nv, zj, ztype, nrhs, 3, nullptr, 0);
      launches += 1 + (P.coarse_m ? 2 : 0) + 1;
      if (mixed) spmv_df(P, reinterpret_cast<const float2*>(zj), reinterpret_cast<float4*>(W.w.p), nrhs, s);
      else spmv(P, P.xi_prob, zj, ztype, W.w.p, nrhs, s);
      ++launches;
      if (P.weighted) {
        // weighted Arnoldi (Sec. 5.2): inner products <v_i, w>_D = v_i^H (D w)
        auto dmul = [&](double2* in, double2* out) {
          if (mixed) dmul_df(P, reinterpret_cast<const float4*>(in), reinterpret_cast<float4*>(out), nrhs, s);
          else spmv_km(P, -P.k * P.k, 0.0, in, 0, out, nrhs, s);
        };
        auto wdots = [&]() {  // h = V^H (D w), entry j+1 = w^H D w
          if (mixed) dots_mixed(W, n, j + 1, 1, s, nullptr, W.r.p, W.w.p);
          else dots(W, n, j + 1, 1, s, W.r.p, W.w.p);
        };
        auto update = [&]() {
          if (mixed)
            orth_update_df(W.nblk, n, nrhs, j + 1, basis_hi(W), basis_lo(W), W.h2.p, W.hs.p,
                           W.active.p, reinterpret_cast<float4*>(W.w.p), W.npart.p, s);
          else
            orth_update(W, n, j + 1, s);
        };
        dmul(W.w.p, W.r.p);
        wdots();
        MX_CUDA(cudaMemcpyAsync(W.h1.p, W.h2.p, (size_t)(j + 2) * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        update();
        dmul(W.w.p, W.r.p);
        wdots();
        {
          ProfScope ps(K_ARNOLDI_SMALL, s);
          MX_LAUNCH(k_arnoldi_finish_w<<<1, 32, 0, s>>>(nrhs, j, m, 0, W.h1.p, W.h2.p, W.H.p, W.active.p, W.flags.p));
          MX_CHECK_LAUNCH();
        }
        MX_CUDA(cudaMemcpyAsync(W.h_flags, W.flags.p, 8, cudaMemcpyDeviceToHost, s));
        MX_CUDA(cudaStreamSynchronize(s));
        if (W.h_flags[1]) {
          update();
          ProfScope ps(K_ARNOLDI_SMALL, s);
          MX_LAUNCH(k_arnoldi_finish_w<<<1, 32, 0, s>>>(nrhs, j, m, 1, W.h1.p, W.h2.p, W.H.p, W.active.p, W.flags.p));
          MX_CHECK_LAUNCH();
        }
        launches += 8;
      }
      if (mixed && !P.weighted) {
        // classical Gram-Schmidt, two passes: c64 inner products, double-float update,
        // double-float inner products, c64 correction fused with the normalisation
        const int nb = std::min(W.nblk, 3 * sm_count());
        float2* Vh = basis_hi(W);
        dots_c64(nb, n, nrhs, j + 1, Vh, reinterpret_cast<const float4*>(W.w.p), W.active.p, W.hpart.p, s);
        {
          ProfScope ps(K_ARNOLDI_SMALL, s);
          MX_LAUNCH(k_reduce_dots<<<grid_for((int64_t)(j + 1) * nrhs * 32, 256), 256, 0, s>>>(nb, j + 1, nrhs, W.hpart.p,
                                                                                           W.h2.p));
          MX_LAUNCH(k_cgs2_finish<<<1, 32, 0, s>>>(W.nblk, nrhs, j, m, 0, W.h2.p, W.npart.p, W.H.p, W.active.p,
                                                  W.g2.p, W.inv2.p));
          MX_CHECK_LAUNCH();
        }
        orth_update_df(W.nblk, n, nrhs, j + 1, Vh, basis_lo(W), W.h2.p, W.hs.p, W.active.p,
                       reinterpret_cast<float4*>(W.w.p), W.npart.p, s);
        dots_mixed(W, n, j + 1, 0, s, P.tune_dots == 0 ? P.status.p + 2 : nullptr);
        {
          ProfScope ps(K_ARNOLDI_SMALL, s);
          MX_LAUNCH(k_cgs2_finish<<<1, 32, 0, s>>>(W.nblk, nrhs, j, m, 1, W.h2.p, W.npart.p, W.H.p, W.active.p,
                                                  W.g2.p, W.inv2.p));
          MX_CHECK_LAUNCH();
        }
        update2_normalize(nv, nrhs, j + 1, Vh, W.g2.p, W.inv2.p, reinterpret_cast<const float4*>(W.w.p),
                          Vh + (int64_t)(j + 1) * nv, basis_lo(W) + (int64_t)(j + 1) * nv, s);
        launches += 9;
      }
      // Arnoldi: classical Gram-Schmidt, second pass when needed
      for (int pass = 0; pass < 2 && !P.weighted && !mixed; ++pass) {
        if (pass == 1) {
          MX_CUDA(cudaMemcpyAsync(W.h_flags, W.flags.p, 8, cudaMemcpyDeviceToHost, s));
          MX_CUDA(cudaStreamSynchronize(s));
          if (!W.h_flags[1]) break;
        }
        dots(W, n, j + 1, pass == 0 ? 1 : 0, s);
        orth_update(W, n, j + 1, s);
        ProfScope ps(K_ARNOLDI_SMALL, s);
        MX_LAUNCH(k_arnoldi_finish<<<1, 32, 0, s>>>(W.nblk, nrhs, j, m, pass, W.h2.p, W.npart.p, W.H.p, W.wnorm0.p,
                                          W.active.p, W.flags.p));
        MX_CHECK_LAUNCH();
        launches += 4;
      }
      if (mixed && P.weighted) {
        normalize_df(nv, nrhs, j, m, W.H.p, W.active.p, reinterpret_cast<const float4*>(W.w.p),
                     basis_hi(W) + (int64_t)(j + 1) * nv, basis_lo(W) + (int64_t)(j + 1) * nv, s);
      } else if (!mixed) {
        ProfScope ps(K_ARNOLDI_SMALL, s, 1, 32.0 * (double)nv, 2.0 * (double)nv);
        MX_LAUNCH(k_normalize<<<gv, 256, 0, s>>>(nv, nrhs, j, m, W.H.p, W.active.p, W.w.p,
                                                 W.V.p + (int64_t)(j + 1) * nv));
      }
      ProfScope ps(K_ARNOLDI_SMALL, s);
      MX_LAUNCH(k_givens<<<1, 32, 0, s>>>(nrhs, j, m, tol, W.bnorm.p, W.H.p, W.cs.p, W.sn.p, W.g.p, W.active.p, W.est.p,
                                W.flags.p));
      MX_CHECK_LAUNCH();
      launches += 2;
      MX_CUDA(cudaMemcpyAsync(W.h_small, W.est.p, nrhs * 8, cudaMemcpyDeviceToHost, s));
      MX_CUDA(cudaStreamSynchronize(s));
      ++total_its;
      bool any = false;
      for (int r = 0; r < nrhs; ++r) {
        if (!act[r]) continue;
        its[r] += 1;
        kcols[r] = j + 1;
        estv[r] = W.h_small[r];
        if (estv[r] <= tol || its[r] >= max_it) act[r] = 0;  // stop this right-hand side
        any = any || act[r];
      }
      MX_CUDA(cudaMemcpyAsync(W.active.p, act.data(), nrhs * 4, cudaMemcpyHostToDevice, s));
      if (!any) break;
    }
    // x += Z y for the right-hand sides that ran in this cycle
    for (int r = 0; r < nrhs; ++r) if (!start_active[r]) kcols[r] = 0;
    MX_CUDA(cudaMemcpyAsync(dk.p, kcols.data(), nrhs * 4, cudaMemcpyHostToDevice, s));
    {
      int kmax = 0;
      for (int r = 0; r < nrhs; ++r) kmax = std::max(kmax, kcols[r]);
      ProfScope ps(K_UPDATE_X, s, mixed ? 3 : 2, ((double)zsz * kmax + 32.0) * (double)nv, 8.0 * kmax * (double)nv);
    MX_LAUNCH(k_backsolve<<<1, 32, 0, s>>>(nrhs, m, dk.p, W.H.p, W.g.p, W.y.p));
    if (mixed) {
      update_x_df(nv, nrhs, kmax, dk.p, (const float2*)W.Z.p, W.y.p, W.hs.p, W.x.p, s);
    } else {
      MX_LAUNCH(k_update_x<double2><<<gv, 256, 0, s>>>(n, nrhs, dk.p, (const double2*)W.Z.p, W.y.p, W.x.p));
      MX_CHECK_LAUNCH();
    }
    }
    true_residual(P, W, s);
    launches += 4;
    // restart set-up for every right-hand side that is not finished
    MX_LAUNCH(k_restart<<<1, 32, 0, s>>>(W.nblk, nrhs, m, W.npart.p, W.bnorm.p, tol, W.active.p, beta.p, W.g.p));
    MX_CHECK_LAUNCH();
    ++launches;
    MX_CUDA(cudaMemcpyAsync(W.h_small, beta.p, nrhs * 8, cudaMemcpyDeviceToHost, s));
    MX_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int r = 0; r < nrhs; ++r) {
      if (done[r]) { act[r] = 0; continue; }
      rel[r] = W.h_small[r] / bn[r];
      if (rel[r] <= tol || its[r] >= max_it) {
        done[r] = 1;
        act[r] = 0;
      } else {
        act[r] = 1;
        any = true;
      }
    }
    // continuous batching: report finished columns, take new right-hand sides into free ones
    while (hook && !P.weighted) {
      std::vector<int> fin;
      for (int r = 0; r < nrhs; ++r)
        if (done[r] && !reported[r]) {
          reported[r] = 1;
          fin.push_back(r);
        }
      const std::vector<int> filled = hook->at_restart(W.x.p, W.b.p, fin, its, rel, estv);
      if (filled.empty()) break;
      std::vector<int32_t> mask(nrhs, 0);
      for (int r : filled) mask[r] = 1;
      DevBuf<int32_t> dmask(nrhs);
      MX_CUDA(cudaMemcpyAsync(dmask.p, mask.data(), nrhs * 4, cudaMemcpyHostToDevice, s));
      MX_LAUNCH(k_zero_cols<<<gv, 256, 0, s>>>(nv, nrhs, dmask.p, W.x.p));
      MX_CHECK_LAUNCH();
      true_residual(P, W, s);  // new columns: r = b
      MX_LAUNCH(k_restart<<<1, 32, 0, s>>>(W.nblk, nrhs, m, W.npart.p, W.bnorm.p, -1.0, W.active.p, beta.p, W.g.p));
      MX_CHECK_LAUNCH();
      launches += 4;
      MX_CUDA(cudaMemcpyAsync(W.h_small, beta.p, nrhs * 8, cudaMemcpyDeviceToHost, s));
      MX_CUDA(cudaStreamSynchronize(s));
      for (int r : filled) {
        bn[r] = W.h_small[r];
        its[r] = 0;
        reported[r] = 0;
        estv[r] = bn[r] > 0 ? 1.0 : 0.0;
        rel[r] = estv[r];
        done[r] = bn[r] > 0 ? 0 : 1;  // a zero right-hand side is done at once (x = 0)
        act[r] = !done[r];
        any = any || act[r];
      }
      MX_CUDA(cudaMemcpyAsync(W.bnorm.p, bn.data(), nrhs * 8, cudaMemcpyHostToDevice, s));
    }
    if (!any) break;
    ++restarts;
    MX_CUDA(cudaMemcpyAsync(W.active.p, act.data(), nrhs * 4, cudaMemcpyHostToDevice, s));
    if (mixed) {
      scale_v0_df(nv, nrhs, beta.p, W.active.p, W.r.p, basis_hi(W), basis_lo(W), s);
    } else {
      MX_LAUNCH(k_scale_v0<<<gv, 256, 0, s>>>(nv, nrhs, beta.p, W.active.p, W.r.p, W.V.p));
      MX_CHECK_LAUNCH();
    }
    ++launches;
  }
  MX_CUDA(cudaMemcpyAsync(x, W.x.p, nv * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  int32_t timeouts = 0;
  MX_CUDA(cudaMemcpyAsync(&timeouts, P.status.p + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  MX_REQUIRE(timeouts == 0, MX_ETIMEOUT, std::to_string(timeouts) + " tensor-core waits ran out in the local solves");
  int rc = MX_OK;
  int maxits = 0;
  for (int r = 0; r < nrhs; ++r) {
    const bool ok = rel[r] <= tol;
    if (!ok) rc = MX_ENOCONV;
    maxits = std::max(maxits, its[r]);
    if (stats) {
      stats[r].iterations = its[r];
      stats[r].converged = ok ? 1 : 0;
      stats[r].rel_residual = rel[r];
      stats[r].rel_estimate = estv[r];
    }
  }
  P.timing.solve_launches = launches;
  P.timing.restarts = restarts;
  P.timing.max_iterations = maxits;
  (void)total_its;
  return rc;
}

}  // namespace mx

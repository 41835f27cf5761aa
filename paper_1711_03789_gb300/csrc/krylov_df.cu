// Krylov kernels of the mixed form in double-float arithmetic (df64.cuh): the operator
// w = A z_j on the stored c64 z_j, the classical Gram-Schmidt passes and the
// normalisation, with the basis V and w stored as complex double-floats (float4
// {re_hi, im_hi, re_lo, im_lo}, 16 bytes like c128). The small dense work (H, Givens,
// least squares), the solution update and the true residual stay in FP64; inner products
// leave the kernels as FP64 block partials.
#include "df64.cuh"
#include "problem.cuh"

namespace mx {

// coef[e] = {a_hi, a_lo, b_hi, b_lo} with a + i b = K_e - (sr + i si) M_e - i bc B_e (B: the
// impedance term, absent with PEC)
__global__ void k_coef_df(int64_t nnz, const double* K, const double* M, double sr, double si, float4* coef,
                          const double* B, double bc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const double im = -si * M[e] - (B ? bc * B[e] : 0.0);
    const float2 a = df::split(K[e] - sr * M[e]), b = df::split(im);
    coef[e] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// w[i][r] = sum_e (a_e + i b_e) z[col_e][r], z c64 (exact FP32 inputs)
__global__ void k_spmv_df(int64_t rows, int nrhs, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const float4* __restrict__ coef, const float2* __restrict__ z, float4* __restrict__ w) {
  const int64_t work = rows * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const int64_t i = t / nrhs;
    df::Acc re, im;
    const int32_t e1 = rowptr[i + 1];
    for (int32_t e = rowptr[i]; e < e1; ++e) {
      const float2 x = z[(int64_t)col[e] * nrhs + r];
      const float4 c = coef[e];
      df::add_prod(re, c.x, c.y, x.x);
      df::add_prod(re, c.z, c.w, -x.y);
      df::add_prod(im, c.x, c.y, x.y);
      df::add_prod(im, c.z, c.w, x.x);
    }
    const float2 a = df::value(re), b = df::value(im);
    w[t] = make_float4(a.x, b.x, a.y, b.y);
  }
}

// hpart[blk][i][r] = sum over the block's rows of conj(V_i[x][r]) w[x][r] (i == nvec:
// |w|^2 when with_norm). Same row split as the update: lanes (xl, r), the block's warps
// stride over its contiguous rows. A lane keeps DOTS_U steps of w in registers and streams
// every basis vector against them, so V and w each leave HBM once (per chunk of DOTS_IC
// basis vectors); the per-step sums are reduced across the row lanes and added into
// warp-private compensated accumulators in shared memory (no block barrier in the loop).
constexpr int DOTS_U = 8;
constexpr int DOTS_IC = 32;
template <int RP>
__global__ void __launch_bounds__(256) k_dots_df(int64_t n, int nrhs, int nvec, int with_norm,
                                                 const float4* __restrict__ V, const float4* __restrict__ w,
                                                 const int32_t* __restrict__ active, double2* __restrict__ hpart,
                                                 const float4* __restrict__ extra) {
  constexpr int XL = 32 / RP;
  extern __shared__ float4 acc_sm[];  // [8 warps][DOTS_IC][RP]: {re_s, re_e, im_s, im_e}
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane % RP, xl = lane / RP;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
  const int total = nvec + with_norm;
  const int64_t nv = n * nrhs;
  const bool on = r < nrhs && active[min(r, nrhs - 1)];
  float4* my = acc_sm + (size_t)warp * DOTS_IC * RP;
  for (int ic = 0; ic < total; ic += DOTS_IC) {
    const int icn = min(DOTS_IC, total - ic);
    for (int t = lane; t < DOTS_IC * RP; t += 32) my[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    for (int64_t xb = x0 + warp * XL; xb < x1; xb += (int64_t)8 * XL * DOTS_U) {
      float4 c[DOTS_U];
#pragma unroll
      for (int u = 0; u < DOTS_U; ++u) {
        const int64_t x = xb + (int64_t)u * 8 * XL + xl;
        c[u] = (on && x < x1) ? w[x * nrhs + r] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int k = 0; k < icn; ++k) {
        const int i = ic + k;
        const float4* Vi = (i < nvec) ? V + (int64_t)i * nv : (extra ? extra : w);
        df::Acc are, aim;
#pragma unroll
        for (int u = 0; u < DOTS_U; ++u) {
          const int64_t x = xb + (int64_t)u * 8 * XL + xl;
          const float4 a = (on && x < x1) ? Vi[x * nrhs + r] : make_float4(0.f, 0.f, 0.f, 0.f);
          // conj(a) c = (a.re c.re + a.im c.im) + i (a.re c.im - a.im c.re)
          df::add_prod2(are, a.x, a.z, c[u].x, c[u].z);
          df::add_prod2(are, a.y, a.w, c[u].y, c[u].w);
          df::add_prod2(aim, a.x, a.z, c[u].y, c[u].w);
          df::add_prod2(aim, -a.y, -a.w, c[u].x, c[u].z);
        }
        // fold the row lanes (same r) together, then into the warp's accumulator
#pragma unroll
        for (int o = RP; o < 32; o <<= 1) {
          float s, e;
          df::two_sum(are.s, __shfl_xor_sync(0xffffffffu, are.s, o), s, e);
          are.e = __fadd_rn(__fadd_rn(are.e, __shfl_xor_sync(0xffffffffu, are.e, o)), e);
          are.s = s;
          df::two_sum(aim.s, __shfl_xor_sync(0xffffffffu, aim.s, o), s, e);
          aim.e = __fadd_rn(__fadd_rn(aim.e, __shfl_xor_sync(0xffffffffu, aim.e, o)), e);
          aim.s = s;
        }
        if (xl == 0) {
          float4 m = my[k * RP + r];
          float s, e;
          df::two_sum(m.x, are.s, s, e);
          m.y = __fadd_rn(m.y, __fadd_rn(are.e, e));
          m.x = s;
          df::two_sum(m.z, aim.s, s, e);
          m.w = __fadd_rn(m.w, __fadd_rn(aim.e, e));
          m.z = s;
          my[k * RP + r] = m;
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < icn * RP; t += blockDim.x) {
      const int k = t / RP, rr = t % RP;
      double sx = 0, sy = 0;
      for (int wq = 0; wq < 8; ++wq) {
        const float4 m = acc_sm[((size_t)wq * DOTS_IC + k) * RP + rr];
        sx += (double)m.x + (double)m.y;
        sy += (double)m.z + (double)m.w;
      }
      if (rr < nrhs) hpart[((int64_t)blockIdx.x * total + ic + k) * nrhs + rr] = make_double2(sx, sy);
    }
    __syncthreads();
  }
}

// hs[i][r] = h[i][r] as a complex double-float
__global__ void k_split_h(int count, const double2* h, float4* hs) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) hs[t] = df::split_c(h[t]);
}

// w[x][r] -= sum_{i < nvec} V_i[x][r] h_i[r]; npart[blk][r] = sum over the block of |w|^2
template <int RP>
__global__ void __launch_bounds__(256) k_orth_update_df(int64_t n, int nrhs, int nvec, const float4* __restrict__ V,
                                                        const float4* __restrict__ hs,
                                                        const int32_t* __restrict__ active, float4* __restrict__ w,
                                                        double* __restrict__ npart) {
  constexpr int XL = 32 / RP;
  __shared__ double sh[8][RP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane % RP, xl = lane / RP;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
  const int64_t nv = n * nrhs;
  const bool on = r < nrhs && active[min(r, nrhs - 1)];
  df::Acc nrm;
  if (on)
    for (int64_t x = x0 + warp * XL + xl; x < x1; x += 8 * XL) {
      df::Acc sre, sim;
#pragma unroll 8
      for (int i = 0; i < nvec; ++i) {
        const float4 a = V[(int64_t)i * nv + x * nrhs + r];
        const float4 c = hs[i * nrhs + r];
        // a c = (a.re c.re - a.im c.im) + i (a.re c.im + a.im c.re)
        df::add_prod2(sre, a.x, a.z, c.x, c.z);
        df::add_prod2(sre, -a.y, -a.w, c.y, c.w);
        df::add_prod2(sim, a.x, a.z, c.y, c.w);
        df::add_prod2(sim, a.y, a.w, c.x, c.z);
      }
      const float4 wv = w[x * nrhs + r];
      const float2 s1 = df::value(sre), s2 = df::value(sim);
      const float2 u = df::sub(wv.x, wv.z, s1.x, s1.y), v = df::sub(wv.y, wv.w, s2.x, s2.y);
      w[x * nrhs + r] = make_float4(u.x, v.x, u.y, v.y);
      df::add_prod2(nrm, u.x, u.y, u.x, u.y);
      df::add_prod2(nrm, v.x, v.y, v.x, v.y);
    }
  double nd = df::to_double(nrm);
#pragma unroll
  for (int o = RP; o < 32; o <<= 1) nd += __shfl_xor_sync(0xffffffffu, nd, o);
  if (xl == 0) sh[warp][r] = nd;
  __syncthreads();
  if (threadIdx.x < RP && threadIdx.x < nrhs) {
    double s = 0;
    for (int wq = 0; wq < 8; ++wq) s += sh[wq][threadIdx.x];
    npart[(int64_t)blockIdx.x * nrhs + threadIdx.x] = s;
  }
}

// v_{j+1} = w / h_{j+1,j}
__global__ void k_normalize_df(int64_t nv, int nrhs, int j, int m, const double2* H, const int32_t* active,
                               const float4* w, float4* vnext) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const double hn = H[((int64_t)j * (m + 1) + j + 1) * nrhs + r].x;
    const float2 inv = df::split((hn > 0 && active[r]) ? 1.0 / hn : 0.0);
    const float4 a = w[t];
    const float2 u = df::mul(a.x, a.z, inv.x, inv.y), v = df::mul(a.y, a.w, inv.x, inv.y);
    vnext[t] = make_float4(u.x, v.x, u.y, v.y);
  }
}

// v0 = r / beta (r FP64)
__global__ void k_scale_v0_df(int64_t nv, int nrhs, const double* beta, const int32_t* active, const double2* r,
                              float4* v0) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % nrhs);
    const double inv = (active[q] && beta[q] > 0) ? 1.0 / beta[q] : 0.0;
    v0[t] = df::split_c(make_double2(r[t].x * inv, r[t].y * inv));
  }
}

// y = A z with y in FP64 (hi + lo of the double-float sums), z c64
__global__ void k_spmv_df_c128(int64_t rows, int nrhs, const int32_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const float4* __restrict__ coef,
                               const float2* __restrict__ z, double2* __restrict__ y) {
  const int64_t work = rows * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const int64_t i = t / nrhs;
    df::Acc re, im;
    const int32_t e1 = rowptr[i + 1];
    for (int32_t e = rowptr[i]; e < e1; ++e) {
      const float2 x = z[(int64_t)col[e] * nrhs + r];
      const float4 c = coef[e];
      df::add_prod(re, c.x, c.y, x.x);
      df::add_prod(re, c.z, c.w, -x.y);
      df::add_prod(im, c.x, c.y, x.y);
      df::add_prod(im, c.z, c.w, x.x);
    }
    y[t] = make_double2(df::to_double(re), df::to_double(im));
  }
}

// y = D w for a real D (coefficients {a_hi, a_lo, 0, 0}), w and y complex double-floats
__global__ void k_dmul_df(int64_t rows, int nrhs, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const float4* __restrict__ coef, const float4* __restrict__ w, float4* __restrict__ y) {
  const int64_t work = rows * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const int64_t i = t / nrhs;
    df::Acc re, im;
    const int32_t e1 = rowptr[i + 1];
    for (int32_t e = rowptr[i]; e < e1; ++e) {
      const float4 x = w[(int64_t)col[e] * nrhs + r];
      const float4 c = coef[e];
      df::add_prod2(re, c.x, c.y, x.x, x.z);
      df::add_prod2(im, c.x, c.y, x.y, x.w);
    }
    const float2 a = df::value(re), b = df::value(im);
    y[t] = make_float4(a.x, b.x, a.y, b.y);
  }
}

// double-float coefficients of A_xi, cached per value of xi (slot 0: xi_prob, 1: xi_prec)
static const float4* coef_df(Problem& P, double xi, int slot, cudaStream_t s) {
  if (P.A_coef_df[slot].n != (size_t)P.A.nnz || P.A_coef_xi[slot] != xi) {
    P.A_coef_df[slot].alloc(P.A.nnz);
    MX_LAUNCH(k_coef_df<<<grid_for(P.A.nnz, 256), 256, 0, s>>>(P.A.nnz, P.A.K.p, P.A.M.p, P.k * P.k, xi,
                                                              P.A_coef_df[slot].p, P.A.B.p, imp_coef(P, xi)));
    MX_CHECK_LAUNCH();
    P.A_coef_xi[slot] = xi;
  }
  return P.A_coef_df[slot].p;
}

// y = D_k w with D_k = K + k^2 M (the weight of weighted GMRES), double-float vectors
void dmul_df(Problem& P, const float4* w, float4* y, int nrhs, cudaStream_t s) {
  if (P.A_coef_df[2].n != (size_t)P.A.nnz) {
    P.A_coef_df[2].alloc(P.A.nnz);
    // K - (sr + i si) M with sr = -k^2, si = 0
    MX_LAUNCH(k_coef_df<<<grid_for(P.A.nnz, 256), 256, 0, s>>>(P.A.nnz, P.A.K.p, P.A.M.p, -P.k * P.k, 0.0,
                                                              P.A_coef_df[2].p, nullptr, 0.0));
    MX_CHECK_LAUNCH();
  }
  const int64_t work = P.A.rows * nrhs;
  ProfScope ps(K_SPMV, s, 1, 20.0 * P.A.nnz + 4.0 * (P.A.rows + 1) + 32.0 * (double)P.A.rows * nrhs,
               4.0 * (double)P.A.nnz * nrhs);
  MX_LAUNCH(k_dmul_df<<<grid_for(work, 256, 152LL * 32), 256, 0, s>>>(P.A.rows, nrhs, P.A.rowptr.p, P.A.col.p,
                                                                      P.A_coef_df[2].p, w, y));
  MX_CHECK_LAUNCH();
}

void spmv_df_c128(Problem& P, double xi, const float2* z, double2* y, int nrhs, cudaStream_t s) {
  const float4* coef = coef_df(P, xi, xi == P.xi_prob ? 0 : 1, s);
  const int64_t work = P.A.rows * nrhs;
  ProfScope ps(K_SPMV, s, 1, 20.0 * P.A.nnz + 4.0 * (P.A.rows + 1) + 24.0 * (double)P.A.rows * nrhs,
               8.0 * (double)P.A.nnz * nrhs);
  MX_LAUNCH(k_spmv_df_c128<<<grid_for(work, 256, 152LL * 32), 256, 0, s>>>(P.A.rows, nrhs, P.A.rowptr.p, P.A.col.p,
                                                                           coef, z, y));
  MX_CHECK_LAUNCH();
}

// ---- host launchers ----------------------------------------------------------------------
void spmv_df(Problem& P, const float2* z, float4* w, int nrhs, cudaStream_t s) {
  const float4* coef = coef_df(P, P.xi_prob, 0, s);
  const int64_t work = P.A.rows * nrhs;
  // coefficients (16 B) and column indices once, z (c64) once, w (16 B) once
  ProfScope ps(K_SPMV, s, 1, 20.0 * P.A.nnz + 4.0 * (P.A.rows + 1) + 24.0 * (double)P.A.rows * nrhs,
               8.0 * (double)P.A.nnz * nrhs);
  MX_LAUNCH(k_spmv_df<<<grid_for(work, 256, 152LL * 32), 256, 0, s>>>(P.A.rows, nrhs, P.A.rowptr.p, P.A.col.p,
                                                                      coef, z, w));
  MX_CHECK_LAUNCH();
}

template <int RP>
static void dots_rp(int nblk, int64_t n, int nrhs, int nvec, int with_norm, const float4* V, const float4* w,
                    const int32_t* active, double2* hpart, cudaStream_t s, const float4* extra) {
  const size_t smem = (size_t)8 * DOTS_IC * RP * sizeof(float4);
  static bool configured = false;
  if (!configured) {
    MX_CUDA(cudaFuncSetAttribute(k_dots_df<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  MX_LAUNCH(k_dots_df<RP><<<nblk, 256, smem, s>>>(n, nrhs, nvec, with_norm, V, w, active, hpart, extra));
}
void dots_df(int nblk, int64_t n, int nrhs, int nvec, int with_norm, const float4* V, const float4* w,
             const int32_t* active, double2* hpart, cudaStream_t s, const float4* extra) {
  ProfScope ps(K_DOTS, s, 1, 16.0 * (nvec + 1) * (double)n * nrhs, 8.0 * (nvec + with_norm) * (double)n * nrhs);
  if (nrhs <= 1) dots_rp<1>(nblk, n, nrhs, nvec, with_norm, V, w, active, hpart, s, extra);
  else if (nrhs <= 2) dots_rp<2>(nblk, n, nrhs, nvec, with_norm, V, w, active, hpart, s, extra);
  else if (nrhs <= 4) dots_rp<4>(nblk, n, nrhs, nvec, with_norm, V, w, active, hpart, s, extra);
  else if (nrhs <= 8) dots_rp<8>(nblk, n, nrhs, nvec, with_norm, V, w, active, hpart, s, extra);
  else if (nrhs <= 16) dots_rp<16>(nblk, n, nrhs, nvec, with_norm, V, w, active, hpart, s, extra);
  else dots_rp<32>(nblk, n, nrhs, nvec, with_norm, V, w, active, hpart, s, extra);
  MX_CHECK_LAUNCH();
}

template <int RP>
static void update_rp(int nblk, int64_t n, int nrhs, int nvec, const float4* V, const float4* hs, const int32_t* active,
                      float4* w, double* npart, cudaStream_t s) {
  MX_LAUNCH(k_orth_update_df<RP><<<nblk, 256, 0, s>>>(n, nrhs, nvec, V, hs, active, w, npart));
}
void orth_update_df(int nblk, int64_t n, int nrhs, int nvec, const float4* V, const double2* h, float4* hs,
                    const int32_t* active, float4* w, double* npart, cudaStream_t s) {
  {
    ProfScope ps(K_ARNOLDI_SMALL, s);
    MX_LAUNCH(k_split_h<<<grid_for((int64_t)nvec * nrhs, 128), 128, 0, s>>>(nvec * nrhs, h, hs));
    MX_CHECK_LAUNCH();
  }
  ProfScope ps(K_ORTH_UPDATE, s, 1, 16.0 * (nvec + 2) * (double)n * nrhs, 8.0 * (nvec + 0.25) * (double)n * nrhs);
  if (nrhs <= 1) update_rp<1>(nblk, n, nrhs, nvec, V, hs, active, w, npart, s);
  else if (nrhs <= 2) update_rp<2>(nblk, n, nrhs, nvec, V, hs, active, w, npart, s);
  else if (nrhs <= 4) update_rp<4>(nblk, n, nrhs, nvec, V, hs, active, w, npart, s);
  else if (nrhs <= 8) update_rp<8>(nblk, n, nrhs, nvec, V, hs, active, w, npart, s);
  else if (nrhs <= 16) update_rp<16>(nblk, n, nrhs, nvec, V, hs, active, w, npart, s);
  else update_rp<32>(nblk, n, nrhs, nvec, V, hs, active, w, npart, s);
  MX_CHECK_LAUNCH();
}

void normalize_df(int64_t nv, int nrhs, int j, int m, const double2* H, const int32_t* active, const float4* w,
                  float4* vnext, cudaStream_t s) {
  ProfScope ps(K_ARNOLDI_SMALL, s, 1, 32.0 * (double)nv, 2.0 * (double)nv);
  MX_LAUNCH(k_normalize_df<<<grid_for(nv, 256), 256, 0, s>>>(nv, nrhs, j, m, H, active, w, vnext));
  MX_CHECK_LAUNCH();
}

void scale_v0_df(int64_t nv, int nrhs, const double* beta, const int32_t* active, const double2* r, float4* v0,
                 cudaStream_t s) {
  MX_LAUNCH(k_scale_v0_df<<<grid_for(nv, 256), 256, 0, s>>>(nv, nrhs, beta, active, r, v0));
  MX_CHECK_LAUNCH();
}

}  // namespace mx

// Coarse level of the two-level preconditioner (Sec. 3.2-3.3, Eq. 3.4 with l = 0):
// the Galerkin matrix A^0_{xi_prec} assembled on the coarse Kuhn mesh, its LU (band-limited,
// no pivoting: A^0 is invertible for xi != 0 by coercivity, Sec. 3.3; FP64 in
// MX_PLAIN_FP64, c64 in MX_MIXED) and the coarse solve y = (A^0)^{-1} R^0 v.
//
// The coarse solve runs as one cooperative kernel: the band triangular sweeps proceed in
// blocks of CB columns; every block of the grid solves the small diagonal triangle
// redundantly, then updates its share of the rows inside the band, and a grid-wide
// barrier separates the steps. In MX_MIXED the factors and the sweep are c64 (the
// preconditioner only needs to be a fixed linear map; the outer FGMRES recurrence stays in
// FP64); in MX_PLAIN_FP64 both are FP64.
#include <cooperative_groups.h>

#include "problem.cuh"

namespace cg = cooperative_groups;

namespace mx {

constexpr int CB = 32;

// bandwidth of the coarse CSR pattern
__global__ void k_csr_band(int64_t rows, const int32_t* rowptr, const int32_t* col, int32_t* out) {
  int bmax = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) bmax = max(bmax, abs((int)(col[e] - i)));
  atomicMax(out, bmax);
}

// A^0 = K_c - (sr + i si) M_c - i bc B_c in band storage (B_c: impedance term, or null)
__global__ void k_coarse_fill(int64_t rows, const int32_t* rowptr, const int32_t* col, const double* K,
                              const double* M, double sr, double si, int b, int ld, double2* A, const double* B,
                              double bc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      A[bidx(0, ld, b, (int)i, col[e])] = make_double2(K[e] - sr * M[e], -si * M[e] - (B ? bc * B[e] : 0.0));
}

__global__ void k_to_c64(int64_t n, const double2* a, float2* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = to_c64(a[i]);
}

// Band LU without pivoting of the single coarse matrix A^0 (Eq. 3.3, l = 0) in one cooperative
// launch instead of three launches per block column. Per block column [k0, k0 + kb): block 0
// factors the diagonal block in shared memory; after a grid-wide barrier every block takes
// rows of L21 = A21 U11^{-1} and columns of U12 = L11^{-1} A12 (one thread each, the 32
// unknowns in registers); after a second barrier the blocks share the 64 x 64 tiles of the
// trailing window A22 -= L21 U12; a third barrier closes the step. The arithmetic of every
// entry is that of the batched per-step kernels (same operations in the same order).
// LU of the kb x kb diagonal block at (k0, k0) by one block in shared memory (no pivoting),
// written back to the band storage; a zero or non-finite pivot counts in *status.
template <typename T2>
__device__ void coarse_diag_block(T2 (*s)[LU_NB + 1], T2* A, int n, int b, int ld, int k0, int32_t* status) {
  constexpr int NB = LU_NB;
  const int tid = threadIdx.x;
  const int kb = min(NB, n - k0);
  for (int t = tid; t < NB * NB; t += blockDim.x) {
    const int i = t % NB, j = t / NB;
    T2 v = czero<T2>();
    if (i < kb && j < kb && abs(i - j) <= b) v = A[bidx(0, ld, b, k0 + i, k0 + j)];
    s[i][j] = v;
  }
  __syncthreads();
  for (int k = 0; k < kb; ++k) {
    const T2 piv = s[k][k];
    const auto p2 = cabs2(piv);
    if (tid == 0 && !(p2 > 0 && p2 < INFINITY)) atomicAdd(status, 1);
    const T2 inv = crcp(piv);
    __syncthreads();
    for (int i = k + 1 + tid; i < kb; i += blockDim.x) s[i][k] = cmul(s[i][k], inv);
    __syncthreads();
    const int w = kb - k - 1;
    for (int t = tid; t < w * w; t += blockDim.x) {
      const int i = k + 1 + t % w, j = k + 1 + t / w;
      T2 v = s[i][j];
      cfms(v, s[i][k], s[k][j]);
      s[i][j] = v;
    }
    __syncthreads();
  }
  for (int t = tid; t < kb * kb; t += blockDim.x) {
    const int i = t % kb, j = t / kb;
    if (abs(i - j) <= b) A[bidx(0, ld, b, k0 + i, k0 + j)] = s[i][j];
  }
  __syncthreads();
}

// Band LU without pivoting of the single coarse matrix A^0 (Eq. 3.3, l = 0) in one cooperative
// launch instead of three launches per block column. Per block column [k0, k0 + kb): every
// block takes rows of L21 = A21 U11^{-1} and columns of U12 = L11^{-1} A12 (one thread each,
// the 32 unknowns in registers); after a grid-wide barrier the blocks share the 64 x 64 tiles
// of the trailing window A22 -= L21 U12, and the next diagonal block -- which lies inside tile
// (0, 0) only -- is factored by block 0 as soon as that tile is done, while the other blocks
// are still updating (look-ahead); a second barrier closes the step. Every entry goes through
// the operations of the batched per-step kernels in the same order.
template <typename T2>
__global__ void __launch_bounds__(256) k_coarse_lu_coop(int n, int b, int ld, T2* A, int32_t* status) {
  constexpr int NB = LU_NB;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char csm[];
  T2(*s)[NB + 1] = reinterpret_cast<T2(*)[NB + 1]>(csm);            // diagonal block
  T2(*sl)[64 + 1] = reinterpret_cast<T2(*)[64 + 1]>(csm);           // update tiles (same space)
  T2(*su)[64 + 1] = reinterpret_cast<T2(*)[64 + 1]>(csm + NB * 65 * sizeof(T2));
  const int tid = threadIdx.x;
  if (blockIdx.x == 0) coarse_diag_block<T2>(s, A, n, b, ld, 0, status);
  grid.sync();
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    const int k1 = k0 + kb;
    const int span = min(n, k1 + b) - k1;
    if (span <= 0) break;  // the last block column (same decision in every block)
    // 1. panels, spread over the grid
    for (int t = tid; t < NB * NB; t += blockDim.x) {
      const int i = t % NB, j = t / NB;
      T2 v = czero<T2>();
      if (i < kb && j < kb && abs(i - j) <= b) v = A[bidx(0, ld, b, k0 + i, k0 + j)];
      s[i][j] = v;
    }
    __syncthreads();
    for (int task = blockIdx.x * blockDim.x + tid; task < 2 * span; task += gridDim.x * blockDim.x) {
      T2 x[NB];
      if (task < span) {
        const int i = k1 + task;
#pragma unroll
        for (int k = 0; k < NB; ++k)
          x[k] = (k < kb && i - (k0 + k) <= b) ? A[bidx(0, ld, b, i, k0 + k)] : czero<T2>();
#pragma unroll
        for (int k = 0; k < NB; ++k) {  // x U11 = a
          if (k < kb) {
            T2 v = x[k];
#pragma unroll
            for (int j = 0; j < k; ++j) cfms(v, x[j], s[j][k]);
            x[k] = cmul(v, crcp(s[k][k]));
          }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < kb && i - (k0 + k) <= b) A[bidx(0, ld, b, i, k0 + k)] = x[k];
      } else {
        const int j = k1 + task - span;
#pragma unroll
        for (int k = 0; k < NB; ++k)
          x[k] = (k < kb && j - (k0 + k) <= b) ? A[bidx(0, ld, b, k0 + k, j)] : czero<T2>();
#pragma unroll
        for (int k = 0; k < NB; ++k) {  // L11 y = a (unit lower)
          if (k < kb) {
            T2 v = x[k];
#pragma unroll
            for (int j2 = 0; j2 < k; ++j2) cfms(v, s[k][j2], x[j2]);
            x[k] = v;
          }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < kb && j - (k0 + k) <= b) A[bidx(0, ld, b, k0 + k, j)] = x[k];
      }
    }
    grid.sync();
    // 2. trailing update, 64 x 64 tiles spread over the grid (256 threads, 4 x 4 outputs each);
    // block 0 takes tile 0 first and then factors the next diagonal block
    __syncthreads();
    const int tiles = (span + 63) / 64;
    for (int tile = blockIdx.x; tile < tiles * tiles; tile += gridDim.x) {
      const int i0 = k1 + 64 * (tile % tiles), j0 = k1 + 64 * (tile / tiles);
      if (i0 - (j0 + 63) <= b && j0 - (i0 + 63) <= b) {  // tile inside the band (uniform)
        for (int t = tid; t < NB * 64; t += blockDim.x) {
          const int r = t % 64, k = t / 64;
          const int i = i0 + r, kk = k0 + k;
          sl[k][r] = (k < kb && i < n && i - kk <= b) ? A[bidx(0, ld, b, i, kk)] : czero<T2>();
          const int j = j0 + r;
          su[k][r] = (k < kb && j < n && j - kk <= b) ? A[bidx(0, ld, b, kk, j)] : czero<T2>();
        }
        __syncthreads();
        const int tx = tid % 16, ty = tid / 16;
        T2 acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = czero<T2>();
        for (int k = 0; k < kb; ++k) {
          T2 lv[4], uv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) lv[a] = sl[k][tx + 16 * a];
#pragma unroll
          for (int c = 0; c < 4; ++c) uv[c] = su[k][ty + 16 * c];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) cfma(acc[a][c], lv[a], uv[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = j0 + ty + 16 * c;
          if (j >= n) continue;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = i0 + tx + 16 * a;
            if (i >= n || abs(i - j) > b) continue;
            T2* p = A + bidx(0, ld, b, i, j);
            *p = csub(*p, acc[a][c]);
          }
        }
        __syncthreads();  // the tile buffers are refilled by the next tile
      }
      if (tile == 0) coarse_diag_block<T2>(s, A, n, b, ld, k1, status);  // look-ahead (block 0)
    }
    grid.sync();
  }
}

template <typename T2>
static void coarse_lu_coop(T2* A, int n, int b, int ld, int32_t* status, cudaStream_t s) {
  const size_t smem = std::max(sizeof(T2) * LU_NB * (LU_NB + 1), sizeof(T2) * 2 * LU_NB * 65);
  static std::atomic<bool> configured{false};
  if (!configured) {
    MX_CUDA(cudaFuncSetAttribute(k_coarse_lu_coop<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  int per_sm = 0;
  MX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_lu_coop<T2>, 256, smem));
  MX_REQUIRE(per_sm > 0, MX_ECUDA, "coarse LU kernel cannot be resident");
  // one block per SM: the 64 x 64 tiles of a step (at most 256) and its 2 span panel tasks
  const int grid = sm_count();
  double flops = 0, bytes = 0;
  for (int k0 = 0; k0 < n; k0 += LU_NB) {
    const double kb = std::min(LU_NB, n - k0);
    const double span = std::max(0, std::min(n, k0 + (int)kb + b) - (k0 + (int)kb));
    flops += 8.0 * span * span * kb + 8.0 * span * kb * kb;
    bytes += sizeof(T2) * (2.0 * span * span + 6.0 * span * kb);
  }
  void* args[] = {(void*)&n, (void*)&b, (void*)&ld, (void*)&A, (void*)&status};
  ProfScope ps(K_COARSE_LU, s, 1, bytes, flops);
  MX_LAUNCH(MX_CUDA(cudaLaunchCooperativeKernel((void*)k_coarse_lu_coop<T2>, grid, 256, args, smem, s)));
}

void factor_coarse(Problem& P) {
  if (!P.coarse_m) return;
  cudaStream_t s = P.stream;
  const int64_t nc = P.coarse.n_dof;
  P.n_c = nc;
  DevBuf<int32_t> bw(1);
  MX_CUDA(cudaMemsetAsync(bw.p, 0, 4, s));
  MX_LAUNCH(k_csr_band<<<grid_for(nc, 256), 256, 0, s>>>(nc, P.Ac.rowptr.p, P.Ac.col.p, bw.p));
  MX_CHECK_LAUNCH();
  int b = 0;
  MX_CUDA(cudaMemcpyAsync(&b, bw.p, 4, cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  P.coarse_band = b;
  P.ld_c = (2 * b + 1 + 3) & ~3;
  P.A0.alloc(P.ld_c * nc);
  MX_CUDA(cudaMemsetAsync(P.A0.p, 0, P.A0.bytes(), s));
  MX_LAUNCH(k_coarse_fill<<<grid_for(nc, 256), 256, 0, s>>>(nc, P.Ac.rowptr.p, P.Ac.col.p, P.Ac.K.p, P.Ac.M.p,
                                                  P.k * P.k, P.xi_prec, b, (int)P.ld_c, P.A0.p, P.Ac.B.p,
                                                  imp_coef(P, P.xi_prec)));
  MX_CHECK_LAUNCH();
  const int32_t meta[3] = {(int32_t)nc, b, (int32_t)P.ld_c};
  const int64_t zero = 0;
  P.c_meta.alloc(3);
  P.c_off.alloc(1);
  MX_CUDA(cudaMemcpyAsync(P.c_meta.p, meta, 12, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(P.c_off.p, &zero, 8, cudaMemcpyHostToDevice, s));
  BandBatch B{1, P.c_meta.p, P.c_meta.p + 1, P.c_meta.p + 2, P.c_off.p};
  const int64_t nq = (nc + CB - 1) / CB;
  if (P.precision == MX_MIXED) {
    // the mixed sweep applies c64 factors: factor the c64 matrix directly (FP32 units,
    // 1/64 of the FP64 work time on this part) and drop the FP64 copy
    P.A0f.alloc(P.A0.n);
    MX_LAUNCH(k_to_c64<<<grid_for(P.A0.n, 256), 256, 0, s>>>(P.A0.n, P.A0.p, P.A0f.p));
    MX_CHECK_LAUNCH();
    MX_CUDA(cudaStreamSynchronize(s));  // the conversion has read A0 before it is released
    P.A0.reset();
    coarse_lu_coop<float2>(P.A0f.p, (int)nc, std::min<int>(b, (int)nc), (int)P.ld_c, P.status.p + 1, s);
    P.c_dinvf.alloc(nq * 2 * CB * CB);
    invert_diag_blocks<float2>(B, P.A0f.p, P.c_off.p, P.c_dinvf.p, (int)nc, s);
    P.A0inv.reset();
    // the inverse's band solve keeps (b + CB) rows of 8 right-hand sides in shared memory
    const bool fits = nc <= COARSE_INVERSE_MAX && (size_t)(b + CB) * 8 * sizeof(float2) <= 200 * 1024;
    if (P.tune_coarse_inverse && fits) {
      MX_CUDA(cudaStreamSynchronize(s));
      P.A0inv.alloc((size_t)nc * nc);
      coarse_inverse(P, P.A0inv.p);
    }
  } else {
    coarse_lu_coop<double2>(P.A0.p, (int)nc, std::min<int>(b, (int)nc), (int)P.ld_c, P.status.p + 1, s);
    P.c_dinv.alloc(nq * 2 * CB * CB);
    invert_diag_blocks<double2>(B, P.A0.p, P.c_off.p, P.c_dinv.p, (int)nc, s);
  }
  MX_CUDA(cudaStreamSynchronize(s));
}

// r0[q][p] = sum_j R^0_pj v[q][j], written as T2: FP64 accumulation for the FP64 form,
// FP32 (values of R^0 in FP32) for the mixed form, whose coarse solve is c64.
template <typename T2, typename AT>
__global__ void k_coarse_restrict(int64_t nc, int64_t n, int nrhs, const int32_t* rowptr, const int32_t* col,
                                  const AT* val, const void* v, int vtype, T2* r0) {
  using A2 = typename cplx<AT>::type;
  const int64_t work = nc * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % nrhs);
    const int64_t p = t / nrhs;
    A2 acc = czero<A2>();
    for (int32_t e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      const int64_t idx = (int64_t)col[e] * nrhs + q;
      A2 x;
      if (vtype == 0) {
        const double2 d = reinterpret_cast<const double2*>(v)[idx];
        x = mk((AT)d.x, (AT)d.y);
      } else if (vtype == 3) {
        const float4 d = reinterpret_cast<const float4*>(v)[idx];
        x = mk((AT)d.x, (AT)d.y);
      } else {
        const float2 d = reinterpret_cast<const float2*>(v)[idx];
        x = mk((AT)d.x, (AT)d.y);
      }
      acc.x = fma(val[e], x.x, acc.x);
      acc.y = fma(val[e], x.y, acc.y);
    }
    r0[p * nrhs + q] = conv<T2>(make_double2(acc.x, acc.y));
  }
}

// entry idx of the vector v read by the restriction: VT 0 c128, 1 c64, 3 complex double-float
// (float4 {re_hi, im_hi, re_lo, im_lo}; its c64 half)
template <typename AT, int VT>
__device__ __forceinline__ typename cplx<AT>::type restrict_load(const void* v, int64_t idx) {
  if constexpr (VT == 0) {
    const double2 d = reinterpret_cast<const double2*>(v)[idx];
    return mk((AT)d.x, (AT)d.y);
  } else if constexpr (VT == 3) {
    const float4 d = reinterpret_cast<const float4*>(v)[idx];
    return mk((AT)d.x, (AT)d.y);
  } else {
    const float2 d = reinterpret_cast<const float2*>(v)[idx];
    return mk((AT)d.x, (AT)d.y);
  }
}

// R^0 v with one block per coarse row (grid-stride): thread (g, q) sums the entries
// rowptr[p] + g, + G, ... of right-hand side q (G = blockDim / nrhs groups), and the G
// partial sums are added in group order (deterministic). A coarse row has several hundred
// entries, so its gathers of v are spread over the whole block instead of one thread; each
// thread issues the gathers of four of its entries before their products (the chain of
// column index and gather is latency-bound otherwise), and adds the products in entry order.
template <typename T2, typename AT, int VT>
__global__ void __launch_bounds__(256) k_coarse_restrict_rows(int64_t nc, int nrhs, const int32_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ col,
                                                              const AT* __restrict__ val, const void* v, T2* r0) {
  using A2 = typename cplx<AT>::type;
  constexpr int U = 4;
  __shared__ A2 part[256];
  const int G = blockDim.x / nrhs;
  const int q = threadIdx.x % nrhs, g = threadIdx.x / nrhs;
  for (int64_t p = blockIdx.x; p < nc; p += gridDim.x) {
    A2 acc = czero<A2>();
    if (g < G) {
      const int32_t e1 = rowptr[p + 1];
      int32_t e = rowptr[p] + g;
      for (; e + (U - 1) * G < e1; e += U * G) {
        int32_t c[U];
        AT w[U];
        A2 x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          c[u] = col[e + u * G];
          w[u] = val[e + u * G];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = restrict_load<AT, VT>(v, (int64_t)c[u] * nrhs + q);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          acc.x = fma(w[u], x[u].x, acc.x);
          acc.y = fma(w[u], x[u].y, acc.y);
        }
      }
      for (; e < e1; e += G) {
        const A2 x = restrict_load<AT, VT>(v, (int64_t)col[e] * nrhs + q);
        acc.x = fma(val[e], x.x, acc.x);
        acc.y = fma(val[e], x.y, acc.y);
      }
    }
    if (g < G) part[g * nrhs + q] = acc;
    __syncthreads();
    if (threadIdx.x < nrhs) {
      A2 s = czero<A2>();
      for (int gg = 0; gg < G; ++gg) {
        s.x += part[gg * nrhs + threadIdx.x].x;
        s.y += part[gg * nrhs + threadIdx.x].y;
      }
      r0[p * nrhs + threadIdx.x] = conv<T2>(make_double2(s.x, s.y));
    }
    __syncthreads();
  }
}

template <typename T2, typename AT>
static void restrict_rows(int64_t nc, int nrhs, const int32_t* rowptr, const int32_t* col, const AT* val,
                          const void* v, int vtype, T2* r0, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<int64_t>(nc, 152LL * 8);
  if (vtype == 0)
    MX_LAUNCH(k_coarse_restrict_rows<T2, AT, 0><<<grid, 256, 0, s>>>(nc, nrhs, rowptr, col, val, v, r0));
  else if (vtype == 3)
    MX_LAUNCH(k_coarse_restrict_rows<T2, AT, 3><<<grid, 256, 0, s>>>(nc, nrhs, rowptr, col, val, v, r0));
  else
    MX_LAUNCH(k_coarse_restrict_rows<T2, AT, 1><<<grid, 256, 0, s>>>(nc, nrhs, rowptr, col, val, v, r0));
}

__global__ void k_to_f32v(int64_t n, const double* a, float* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Band triangular sweeps on r [n][nrhs] (in place): forward with unit lower L, backward
// with upper U. Grid-wide barriers between column blocks.
template <typename T2>
__global__ void k_coarse_sweep(int n, int b, int ld, const T2* F, const T2* Dinv, T2* r, int nrhs) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ unsigned char smem_raw[];
  T2* x = reinterpret_cast<T2*>(smem_raw);  // [CB][nrhs]
  __shared__ T2 D[CB][CB + 1];              // diagonal block of the current step
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nblk = (n + CB - 1) / CB;
  for (int t = tid; t < CB * nrhs; t += nt) x[t] = czero<T2>();
  __syncthreads();
  for (int dir = 0; dir < 2; ++dir) {  // 0: forward (unit lower L), 1: backward (upper U)
    for (int s = 0; s < nblk; ++s) {
      const int blk = dir == 0 ? s : nblk - 1 - s;
      const int c0 = blk * CB, c1 = min(n, c0 + CB), kb = c1 - c0;
      for (int t = tid; t < kb * nrhs; t += nt) x[t] = r[(int64_t)c0 * nrhs + t];
      __syncthreads();
      // every block applies the inverted diagonal block redundantly: x_blk = D r_blk
      {
        const T2* Dq = Dinv + (int64_t)blk * 2 * CB * CB + (dir == 0 ? 0 : CB * CB);  // column-major
        for (int t = tid; t < CB * CB; t += nt) D[t % CB][t / CB] = Dq[t];
        __syncthreads();
        T2 out[4];
        for (int c = 0; c < 4; ++c) {
          const int t = tid + nt * c;
          out[c] = czero<T2>();
          if (t < kb * nrhs) {
            const int i = t / nrhs, q = t % nrhs;
            const int k0 = dir == 0 ? 0 : i, k1 = dir == 0 ? i + 1 : kb;
            for (int k = k0; k < k1; ++k) cfma(out[c], D[i][k], x[k * nrhs + q]);
          }
        }
        __syncthreads();
        for (int c = 0; c < 4; ++c) {
          const int t = tid + nt * c;
          if (t < kb * nrhs) x[t] = out[c];
        }
      }
      __syncthreads();
      if (blockIdx.x == 0)
        for (int t = tid; t < kb * nrhs; t += nt) r[(int64_t)c0 * nrhs + t] = x[t];
      // rows inside the band outside the block
      const int r0 = dir == 0 ? c1 : max(0, c0 - b);
      const int r1 = dir == 0 ? min(n, c1 + b) : c0;
      const int64_t work = (int64_t)(r1 - r0) * nrhs;
      for (int64_t t = blockIdx.x * (int64_t)nt + tid; t < work; t += (int64_t)gridDim.x * nt) {
        const int i = r0 + (int)(t / nrhs), q = (int)(t % nrhs);
        T2 acc = r[(int64_t)i * nrhs + q];
        const int k0 = dir == 0 ? max(c0, i - b) : c0;
        const int k1 = dir == 0 ? c1 : min(c1, i + b + 1);
        // fixed trip count, all factor loads issued ahead (out-of-range entries load as 0;
        // x rows past kb are zero-initialised)
        T2 f[CB];
#pragma unroll
        for (int u = 0; u < CB; ++u) {
          const int k = c0 + u;
          f[u] = (k >= k0 && k < k1) ? F[bidx(0, ld, b, i, k)] : czero<T2>();
        }
#pragma unroll
        for (int u = 0; u < CB; ++u) cfms(acc, f[u], x[u * nrhs + q]);
        r[(int64_t)i * nrhs + q] = acc;
      }
      grid.sync();
    }
  }
}

template <typename T2>
static void sweep(Problem& P, T2* F, const T2* Dinv, T2* r, int nrhs) {
  const int n = (int)P.n_c, b = P.coarse_band, ld = (int)P.ld_c;
  const size_t smem = (size_t)CB * nrhs * sizeof(T2);
  MX_REQUIRE(nrhs <= 32 && smem <= 48 * 1024, MX_EINVAL, "too many right-hand sides for the coarse sweep");
  int per_sm = 0;
  MX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_sweep<T2>, 256, smem));
  MX_REQUIRE(per_sm > 0, MX_ECUDA, "coarse sweep kernel cannot be resident");
  const int64_t work = (int64_t)std::min(b, n) * nrhs;
  int grid = (int)std::min<int64_t>((int64_t)sm_count() * per_sm, std::max<int64_t>(1, (work + 255) / 256));
  grid = std::max(1, std::min(grid, sm_count()));
  // fewer blocks make the grid-wide barrier between column blocks cheaper (tunable)
  if (P.tune_coarse_blocks > 0) grid = std::min(P.tune_coarse_blocks, sm_count() * per_sm);
  void* args[] = {(void*)&n, (void*)&b, (void*)&ld, (void*)&F, (void*)&Dinv, (void*)&r, (void*)&nrhs};
  const double entries = (double)n * (2.0 * b + 1.0) - (double)b * (b + 1.0);
  ProfScope ps(K_COARSE_SWEEP, P.stream, 1, sizeof(T2) * (entries + 2.0 * n * nrhs), 8.0 * entries * nrhs);
  MX_LAUNCH(MX_CUDA(cudaLaunchCooperativeKernel((void*)k_coarse_sweep<T2>, grid, 256, args, smem, P.stream)));
}

// Dense coarse apply with the explicit inverse (mixed form): part[ks][i][r] =
// sum_{j in chunk ks} X[j][i] rc[j][r] (X symmetric, read along rows j). A thread owns two
// adjacent columns i and up to 16 right-hand sides, so a block reads 4 KB of each row of
// X contiguously and X leaves HBM once; the right-hand-side values are broadcast from L1.
constexpr int CD_R = 16;
__global__ void __launch_bounds__(256, 2) k_coarse_dense(int n, int nrhs, int jchunk, const float2* __restrict__ X,
                                                         const float2* __restrict__ rc, float2* __restrict__ part) {
  const int i0 = (blockIdx.x * 256 + threadIdx.x) * 2;
  const int g0 = blockIdx.z * CD_R;
  const int gn = min(CD_R, nrhs - g0);
  const int j0 = blockIdx.y * jchunk, j1 = min(n, j0 + jchunk);
  if (i0 >= n || gn <= 0) return;
  const bool two = i0 + 1 < n;
  float2 acc0[CD_R], acc1[CD_R];
#pragma unroll
  for (int g = 0; g < CD_R; ++g) acc0[g] = acc1[g] = make_float2(0.f, 0.f);
  const bool vec = gn == CD_R && (nrhs % 2) == 0;
  // the two columns as one 16-byte load when the row offset is even
  const bool pair = two && (n % 2) == 0;
  constexpr int JU = 8;  // rows of X in flight per thread
  for (int jb = j0; jb < j1; jb += JU) {
    float2 xa[JU], xb[JU];
#pragma unroll
    for (int u = 0; u < JU; ++u) {
      const int j = jb + u;
      xa[u] = xb[u] = make_float2(0.f, 0.f);
      if (j < j1) {
        const float2* xr = X + (int64_t)j * n + i0;
        if (pair) {
          const float4 q = *reinterpret_cast<const float4*>(xr);
          xa[u] = make_float2(q.x, q.y);
          xb[u] = make_float2(q.z, q.w);
        } else {
          xa[u] = xr[0];
          if (two) xb[u] = xr[1];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < JU; ++u) {
      const int j = jb + u;
      if (j >= j1) break;
      const float2* r = rc + (int64_t)j * nrhs + g0;
      if (vec) {
        const float4* r4 = reinterpret_cast<const float4*>(r);
#pragma unroll
        for (int g = 0; g < CD_R / 2; ++g) {
          const float4 q = r4[g];
          cfma(acc0[2 * g], xa[u], make_float2(q.x, q.y));
          cfma(acc1[2 * g], xb[u], make_float2(q.x, q.y));
          cfma(acc0[2 * g + 1], xa[u], make_float2(q.z, q.w));
          cfma(acc1[2 * g + 1], xb[u], make_float2(q.z, q.w));
        }
      } else {
#pragma unroll
        for (int g = 0; g < CD_R; ++g)
          if (g < gn) {
            const float2 q = r[g];
            cfma(acc0[g], xa[u], q);
            cfma(acc1[g], xb[u], q);
          }
      }
    }
  }
  float2* o = part + ((int64_t)blockIdx.y * n + i0) * nrhs + g0;
#pragma unroll
  for (int g = 0; g < CD_R; ++g)
    if (g < gn) {
      o[g] = acc0[g];
      if (two) o[nrhs + g] = acc1[g];
    }
}

__global__ void k_coarse_sum(int64_t count, int ks, const float2* part, float2* y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < ks; ++k) {
      const float2 v = part[(int64_t)k * count + t];
      s.x += v.x;
      s.y += v.y;
    }
    y[t] = s;
  }
}

__global__ void k_c128_to_c64(int64_t count, const double2* a, float2* b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = make_float2((float)a[t].x, (float)a[t].y);
}

// FP32 copy of the R^0 values (mixed-form restriction), made on first use
static const float* r0_valf(Problem& P) {
  if (P.R0_valf.n != (size_t)P.R0.nnz) {
    P.R0_valf.alloc(P.R0.nnz);
    MX_LAUNCH(k_to_f32v<<<grid_for(P.R0.nnz, 256), 256, 0, P.stream>>>(P.R0.nnz, P.R0.val.p, P.R0_valf.p));
    MX_CHECK_LAUNCH();
  }
  return P.R0_valf.p;
}

// Inexact coarse solve (Sec. 6.4): y = result of the inner GMRES on A^0 y = R^0 v (y0 = 0,
// relative tolerance c_tol, at most c_max_it iterations, unrestarted), preconditioned by the
// inner problem's one-level Schwarz method. R^0 v is formed in FP64 (FP32 products in the
// mixed form, whose coarse solve is c64 anyway); the inner iteration runs in the handle's
// precision; a solution that misses c_tol after c_max_it iterations is used as it is. The
// inner kernels are booked under coarse_gmres.
static void coarse_solve_inner(Problem& P, const void* v, int vtype, double2* yc, int nrhs, double rb) {
  cudaStream_t s = P.stream;
  const int64_t nc = P.n_c;
  P.c_rhs.ensure((size_t)nc * nrhs);
  P.c_sol.ensure((size_t)nc * nrhs);
  {
    ProfScope ps(K_COARSE_RESTRICT, s, 1, rb, 4.0 * P.R0.nnz * nrhs);
    if (P.precision == MX_MIXED)
      MX_LAUNCH(k_coarse_restrict<double2, float><<<grid_for(nc * nrhs, 256), 256, 0, s>>>(
          nc, P.fine.n_dof, nrhs, P.R0.rowptr.p, P.R0.col.p, r0_valf(P), v, vtype, P.c_rhs.p));
    else
      MX_LAUNCH(k_coarse_restrict<double2, double><<<grid_for(nc * nrhs, 256), 256, 0, s>>>(
          nc, P.fine.n_dof, nrhs, P.R0.rowptr.p, P.R0.col.p, P.R0.val.p, v, vtype, P.c_rhs.p));
    MX_CHECK_LAUNCH();
  }
  Problem& Q = *P.coarse_inner;
  Q.stream = s;
  const int saved = prof_redirect(K_COARSE_GMRES);
  try {
    (void)gmres_solve(Q, P.c_rhs.p, P.c_sol.p, nrhs, P.c_tol, 0, P.c_max_it, nullptr);  // MX_ENOCONV allowed
  } catch (...) {
    prof_redirect(saved);
    throw;
  }
  prof_redirect(saved);
  P.timing.coarse_inner_iterations += Q.timing.max_iterations;
  ++P.timing.coarse_inner_solves;
  if (P.precision == MX_MIXED) {
    MX_LAUNCH(k_c128_to_c64<<<grid_for(nc * nrhs, 256), 256, 0, s>>>(nc * nrhs, P.c_sol.p, reinterpret_cast<float2*>(yc)));
    MX_CHECK_LAUNCH();
  } else {
    MX_CUDA(cudaMemcpyAsync(yc, P.c_sol.p, (size_t)nc * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  }
}

void coarse_solve(Problem& P, const void* v, int vtype, double2* yc, int nrhs) {
  cudaStream_t s = P.stream;
  const int64_t nc = P.n_c;
  // unique bytes: R^0 (12 B per entry, row pointers), the input block read once (every fine
  // DOF has a nonzero column in R^0) and the output once; the repeated gathers of v hit L2
  const double vb = vtype == 1 ? 8.0 : 16.0, ob = P.precision == MX_MIXED ? 8.0 : 16.0;
  const double rb = 12.0 * P.R0.nnz + 4.0 * (nc + 1) + vb * (double)P.fine.n_dof * nrhs + ob * nc * nrhs;
  if (P.coarse_inner) {
    coarse_solve_inner(P, v, vtype, yc, nrhs, rb);
    return;
  }
  MX_REQUIRE(P.coarse_factored, MX_ENOTFACTORED, "the direct coarse factors are not built");
  const bool mixed = P.precision == MX_MIXED;
  const bool dense = mixed && P.A0inv.p;
  float2* rf = reinterpret_cast<float2*>(yc);  // c64 view of the workspace (mixed): the coarse solution
  // with the explicit inverse the restriction goes to the upper half of the workspace
  float2* rin = dense ? rf + nc * nrhs : rf;
  {
    ProfScope ps(K_COARSE_RESTRICT, s, 1, rb, 4.0 * P.R0.nnz * nrhs);
    if (mixed)
      restrict_rows<float2, float>(nc, nrhs, P.R0.rowptr.p, P.R0.col.p, r0_valf(P), v, vtype, rin, s);
    else
      restrict_rows<double2, double>(nc, nrhs, P.R0.rowptr.p, P.R0.col.p, P.R0.val.p, v, vtype, yc, s);
    MX_CHECK_LAUNCH();
  }
  if (dense && P.tune_coarse_inverse != 2 && nc % 2 == 0) {
    // tensor cores (3 x TF32): column pairs of X start 16-byte aligned when n_c is even
    ProfScope ps(K_COARSE_SWEEP, s, 1, 8.0 * (double)nc * nc + 8.0 * nc * nrhs * 2.0, 8.0 * (double)nc * nc * nrhs);
    float2* part = nullptr;
    int ks = 0;
    if (coarse_dense_tc(P, rin, nrhs, part, ks)) {
      MX_LAUNCH(k_coarse_sum<<<grid_for(nc * nrhs, 256), 256, 0, s>>>(nc * nrhs, ks, part, rf));
      MX_CHECK_LAUNCH();
      return;
    }
  }
  if (dense) {
    // split the rows of X among ks chunks so that the grid fits in one wave of two blocks
    // per SM (a second, nearly empty wave would double the time)
    const int rows_blocks = (int)((nc + 511) / 512);
    const int zgroups = (nrhs + CD_R - 1) / CD_R;
    const int ks = std::max(1, std::min(64, (2 * sm_count()) / (rows_blocks * zgroups)));
    const int jchunk = (int)((nc + ks - 1) / ks);
    P.c_part.ensure((size_t)ks * nc * nrhs);
    {
      ProfScope ps(K_COARSE_SWEEP, s, 1, 8.0 * (double)nc * nc + 8.0 * nc * nrhs * (1.0 + ks),
                   8.0 * (double)nc * nc * nrhs);
      MX_LAUNCH(k_coarse_dense<<<dim3(rows_blocks, ks, zgroups), 256, 0, s>>>((int)nc, nrhs, jchunk, P.A0inv.p, rin,
                                                                             P.c_part.p));
      MX_CHECK_LAUNCH();
      MX_LAUNCH(k_coarse_sum<<<grid_for(nc * nrhs, 256), 256, 0, s>>>(nc * nrhs, ks, P.c_part.p, rf));
      MX_CHECK_LAUNCH();
    }
    return;
  }
  if (mixed) sweep<float2>(P, P.A0f.p, P.c_dinvf.p, rf, nrhs);
  else sweep<double2>(P, P.A0.p, P.c_dinv.p, yc, nrhs);
}

}  // namespace mx

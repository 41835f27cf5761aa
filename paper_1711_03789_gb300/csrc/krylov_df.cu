// Krylov kernels of the mixed form in double-float arithmetic (df64.cuh): the operator
// w = A z_j on the stored c64 z_j, the classical Gram-Schmidt passes and the
// normalisation. w is a complex double-float vector (float4 {re_hi, im_hi, re_lo, im_lo});
// the basis V is stored as two c64 planes, Vh (the c64 rounding of each entry) and Vl (the
// remainder), so that the passes that need only c64 accuracy read half the bytes. The
// small dense work (H, Givens, least squares), the solution update and the true residual
// stay in FP64; inner products leave the kernels as FP64 block partials.
//
// Arnoldi step (classical Gram-Schmidt, two passes, Sec. 6.1 leaves the orthogonalisation
// open): pass 1 takes h1 = V^H w from the c64 planes (k_dots_c64; its error, about 1e-7 of
// ||w||, is what pass 2 removes), w' = w - V h1 in double-float (k_orth_update_df), pass 2
// h2 = V^H w' in double-float (k_dots_df), and v_{j+1} = (w' - V h2) / ||w''|| with the
// correction V h2 -- of the size of the pass-1 error -- in c64 products on Vh, and
// ||w''||^2 = ||w'||^2 - |h2|^2 (k_update2_normalize).
#include "df64.cuh"
#include "problem.cuh"
#include "tc.cuh"

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

// The same product for an even number of right-hand sides: one thread per (row, pair of
// right-hand sides), so the column index and the coefficients of a nonzero are loaded once for
// two right-hand sides and z is gathered with 16-byte loads; every right-hand side gets the
// same operations in the same order as in k_spmv_df.
__global__ void k_spmv_df2(int64_t rows, int nrhs, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const float4* __restrict__ coef, const float4* __restrict__ z, float4* __restrict__ w) {
  const int half = nrhs / 2;
  const int64_t work = rows * half;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work; t += (int64_t)gridDim.x * blockDim.x) {
    const int r2 = (int)(t % half);
    const int64_t i = t / half;
    df::Acc re0, im0, re1, im1;
    const int32_t e1 = rowptr[i + 1];
    for (int32_t e = rowptr[i]; e < e1; ++e) {
      const float4 x = z[(int64_t)col[e] * half + r2];  // (re, im) of right-hand sides 2 r2, 2 r2 + 1
      const float4 c = coef[e];
      df::add_prod(re0, c.x, c.y, x.x);
      df::add_prod(re0, c.z, c.w, -x.y);
      df::add_prod(im0, c.x, c.y, x.y);
      df::add_prod(im0, c.z, c.w, x.x);
      df::add_prod(re1, c.x, c.y, x.z);
      df::add_prod(re1, c.z, c.w, -x.w);
      df::add_prod(im1, c.x, c.y, x.w);
      df::add_prod(im1, c.z, c.w, x.z);
    }
    const float2 a0 = df::value(re0), b0 = df::value(im0), a1 = df::value(re1), b1 = df::value(im1);
    w[i * nrhs + 2 * r2] = make_float4(a0.x, b0.x, a0.y, b0.y);
    w[i * nrhs + 2 * r2 + 1] = make_float4(a1.x, b1.x, a1.y, b1.y);
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
__global__ void __launch_bounds__(256, 3) k_dots_df(int64_t n, int nrhs, int nvec, int with_norm,
                                                 const float2* __restrict__ Vh, const float2* __restrict__ Vl,
                                                 const float4* __restrict__ w, const int32_t* __restrict__ active,
                                                 double2* __restrict__ hpart, const float4* __restrict__ extra) {
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
        const bool basis = i < nvec;
        const float2* Hi = Vh + (int64_t)i * nv;
        const float2* Lo = Vl + (int64_t)i * nv;
        const float4* Ei = extra ? extra : w;
        df::Acc are, aim;
#pragma unroll
        for (int u = 0; u < DOTS_U; ++u) {
          const int64_t x = xb + (int64_t)u * 8 * XL + xl;
          float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
          if (on && x < x1) {
            if (basis) {
              const float2 ah = Hi[x * nrhs + r], al = Lo[x * nrhs + r];
              a = make_float4(ah.x, ah.y, al.x, al.y);
            } else {
              a = Ei[x * nrhs + r];
            }
          }
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

// Paired form of k_dots_df for an even number of right-hand sides: a lane takes the pair
// (r, r+1), so each plane is read with one 16-byte load per two entries (the c64 planes of
// two neighbouring right-hand sides are adjacent) instead of two 8-byte loads per entry.
// Lanes (xl, rp), rp = pair index fastest; XL2 = 32 / (RP / 2) rows per warp step.
constexpr int DOTS_U2 = 4;

// named barrier of the staged kernel's four consumer warps (the producer warp does not join)
__device__ __forceinline__ void bar_consumers() { tc::bar_sync(1, 128); }

// a += the accumulator of lane (lane ^ o), compensated
__device__ __forceinline__ void fold_lanes(df::Acc& a, int o) {
  float sm, e;
  df::two_sum(a.s, __shfl_xor_sync(0xffffffffu, a.s, o), sm, e);
  a.e = __fadd_rn(__fadd_rn(a.e, __shfl_xor_sync(0xffffffffu, a.e, o)), e);
  a.s = sm;
}
template <int RP>
__global__ void __launch_bounds__(256, 3) k_dots_df2(int64_t n, int nrhs, int nvec, int with_norm,
                                                  const float2* __restrict__ Vh, const float2* __restrict__ Vl,
                                                  const float4* __restrict__ w, const int32_t* __restrict__ active,
                                                  double2* __restrict__ hpart, const float4* __restrict__ extra) {
  constexpr int RP2 = RP / 2;
  constexpr int XL = 32 / RP2;
  extern __shared__ float4 acc_sm2[];  // [8 warps][DOTS_IC][RP]: {re_s, re_e, im_s, im_e}
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rp = lane % RP2, xl = lane / RP2;
  const int r0 = 2 * rp;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
  const int total = nvec + with_norm;
  const int64_t nv = n * nrhs;
  const bool in = r0 < nrhs;  // nrhs even: r0 + 1 < nrhs too
  const bool on0 = in && active[min(r0, nrhs - 1)], on1 = in && active[min(r0 + 1, nrhs - 1)];
  float4* my = acc_sm2 + (size_t)warp * DOTS_IC * RP;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int ic = 0; ic < total; ic += DOTS_IC) {
    const int icn = min(DOTS_IC, total - ic);
    for (int t = lane; t < DOTS_IC * RP; t += 32) my[t] = zero;
    __syncwarp();
    for (int64_t xb = x0 + warp * XL; xb < x1; xb += (int64_t)8 * XL * DOTS_U2) {
      float4 c0[DOTS_U2], c1[DOTS_U2];
#pragma unroll
      for (int u = 0; u < DOTS_U2; ++u) {
        const int64_t x = xb + (int64_t)u * 8 * XL + xl;
        const bool ok = in && x < x1;
        c0[u] = (ok && on0) ? w[x * nrhs + r0] : zero;
        c1[u] = (ok && on1) ? w[x * nrhs + r0 + 1] : zero;
      }
      for (int k = 0; k < icn; ++k) {
        const int i = ic + k;
        const bool basis = i < nvec;
        const float4* Hi = reinterpret_cast<const float4*>(Vh + (int64_t)i * nv);
        const float4* Lo = reinterpret_cast<const float4*>(Vl + (int64_t)i * nv);
        const float4* Ei = extra ? extra : w;
        df::Acc are0, aim0, are1, aim1;
#pragma unroll
        for (int u = 0; u < DOTS_U2; ++u) {
          const int64_t x = xb + (int64_t)u * 8 * XL + xl;
          float4 a0 = zero, a1 = zero;
          if (in && x < x1) {
            if (basis) {
              const int64_t q = (x * nrhs + r0) >> 1;
              const float4 h = Hi[q], l = Lo[q];
              a0 = make_float4(h.x, h.y, l.x, l.y);
              a1 = make_float4(h.z, h.w, l.z, l.w);
            } else {
              a0 = Ei[x * nrhs + r0];
              a1 = Ei[x * nrhs + r0 + 1];
            }
          }
          // conj(a) c = (a.re c.re + a.im c.im) + i (a.re c.im - a.im c.re)
          df::add_prod2(are0, a0.x, a0.z, c0[u].x, c0[u].z);
          df::add_prod2(are0, a0.y, a0.w, c0[u].y, c0[u].w);
          df::add_prod2(aim0, a0.x, a0.z, c0[u].y, c0[u].w);
          df::add_prod2(aim0, -a0.y, -a0.w, c0[u].x, c0[u].z);
          df::add_prod2(are1, a1.x, a1.z, c1[u].x, c1[u].z);
          df::add_prod2(are1, a1.y, a1.w, c1[u].y, c1[u].w);
          df::add_prod2(aim1, a1.x, a1.z, c1[u].y, c1[u].w);
          df::add_prod2(aim1, -a1.y, -a1.w, c1[u].x, c1[u].z);
        }
        // fold the row lanes (same pair) together, then into the warp's accumulators
#pragma unroll
        for (int o = RP2; o < 32; o <<= 1) {
          fold_lanes(are0, o);
          fold_lanes(aim0, o);
          fold_lanes(are1, o);
          fold_lanes(aim1, o);
        }
        if (xl == 0 && in) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const df::Acc& ar = q ? are1 : are0;
            const df::Acc& ai = q ? aim1 : aim0;
            float4 m = my[k * RP + r0 + q];
            float sm, e;
            df::two_sum(m.x, ar.s, sm, e);
            m.y = __fadd_rn(m.y, __fadd_rn(ar.e, e));
            m.x = sm;
            df::two_sum(m.z, ai.s, sm, e);
            m.w = __fadd_rn(m.w, __fadd_rn(ai.e, e));
            m.z = sm;
            my[k * RP + r0 + q] = m;
          }
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < icn * RP; t += blockDim.x) {
      const int k = t / RP, rr = t % RP;
      double sx = 0, sy = 0;
      for (int wq = 0; wq < 8; ++wq) {
        const float4 m = acc_sm2[((size_t)wq * DOTS_IC + k) * RP + rr];
        sx += (double)m.x + (double)m.y;
        sy += (double)m.z + (double)m.w;
      }
      if (rr < nrhs) hpart[((int64_t)blockIdx.x * total + ic + k) * nrhs + rr] = make_double2(sx, sy);
    }
    __syncthreads();
  }
}

// Staged form of the double-float inner products (no norm entry) for nrhs in {2, 4, 8, 16, 32}.
// A producer warp streams the basis through a ring of DS_STAGES shared-memory stages with bulk
// copies, so the loads are in flight while four consumer warps compute. A stage holds DS_VG
// basis vectors (both planes) over XS = 128 / (nrhs / 2) consecutive rows: 32 KB in 2 KB
// copies. Consumer thread (xs, p) takes row xs of every stage and right-hand sides 2p, 2p+1,
// and keeps the 4 * DS_VG compensated accumulators of its chunk of vectors in registers over
// all of its block's rows (w straight from global memory, one row ahead); the row lanes are
// folded once per chunk, not once per row step as in the lane-parallel kernels. Vectors beyond
// DS_VG: the rows are swept again for the next chunk (w read once per chunk). Writes the same
// per-block partials as k_dots_df.
constexpr int DS_VG = 8;                          // basis vectors per stage
constexpr int DS_STAGES = 3;                      // ring depth
constexpr int DS_CONSUMERS = 128;                 // 4 warps
constexpr int DS_THREADS = DS_CONSUMERS + 32;     // + the producer warp
constexpr int DS_TILE = DS_CONSUMERS * 2 * 8;     // one plane of one vector: XS rows x nrhs x 8 B
constexpr int DS_STAGE_BYTES = 2 * DS_VG * DS_TILE;
constexpr int DS_WAIT_LIMIT = 1 << 22;

__global__ void __launch_bounds__(DS_THREADS, 2) k_dots_df_staged(int64_t n, int nrhs, int nvec,
                                                                const float2* __restrict__ Vh,
                                                                const float2* __restrict__ Vl,
                                                                const float4* __restrict__ w,
                                                                const int32_t* __restrict__ active,
                                                                double2* __restrict__ hpart, int32_t* timeout) {
  extern __shared__ __align__(128) unsigned char ds_smem[];
  __shared__ __align__(8) uint64_t full[DS_STAGES], empty[DS_STAGES];
  __shared__ double2 red[DS_CONSUMERS / 32][DS_VG][16][2];  // per-warp folded partials
  __shared__ volatile int stop;
  const int np = nrhs / 2, xsn = DS_CONSUMERS / np;  // pairs per row, rows per stage
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = min(n, (int64_t)blockIdx.x * chunk), x1 = min(n, x0 + chunk);
  const int64_t nv = n * nrhs;
  const uint32_t base = tc::smem_u32(ds_smem);
  const uint32_t full_a = tc::smem_u32(&full[0]), empty_a = tc::smem_u32(&empty[0]);
  if (tid == 0) {
    for (int i = 0; i < DS_STAGES; ++i) {
      tc::mbar_init(full_a + 8 * i, 1);
      tc::mbar_init(empty_a + 8 * i, DS_CONSUMERS / 32);
    }
    tc::mbar_fence_init();
    stop = 0;
  }
  __syncthreads();

  if (warp == DS_CONSUMERS / 32) {
    // producer: stages in the consumers' order (chunk of vectors, row step)
    int64_t st = 0;  // stages issued
    bool ok = true;
    for (int k0 = 0; k0 < nvec && ok; k0 += DS_VG) {
      const int nk = min(DS_VG, nvec - k0);
      for (int64_t x = x0; x < x1 && ok; x += xsn, ++st) {
        const int slot = (int)(st % DS_STAGES), use = (int)(st / DS_STAGES);
        const uint32_t rb = (uint32_t)min((int64_t)xsn, x1 - x) * nrhs * 8;
        if (lane == 0) {
          if (use > 0 && !tc::mbar_wait_flag(empty_a + 8 * slot, (use - 1) & 1, DS_WAIT_LIMIT, &stop)) {
            atomicAdd(timeout, 1);
            stop = 1;
          }
          if (!stop) tc::mbar_expect_tx(full_a + 8 * slot, 2 * nk * rb);
        }
        ok = __shfl_sync(0xffffffffu, stop == 0, 0);
        if (!ok) break;
        if (lane < 2 * nk) {
          const int plane = lane / nk, v = lane % nk;
          const float2* src = (plane ? Vl : Vh) + (int64_t)(k0 + v) * nv + x * nrhs;
          tc::bulk_g2s(base + (uint32_t)slot * DS_STAGE_BYTES + (uint32_t)(plane * DS_VG + v) * DS_TILE, src, rb,
                       full_a + 8 * slot);
        }
      }
    }
    // every copy this block issued lands before the block's shared memory is released: wait
    // for the last phase each slot was given
    if (lane == 0)
      for (int i = 0; i < DS_STAGES && i < st; ++i) {
        const int last = (int)((st - 1 - i) / DS_STAGES);
        if (!tc::mbar_wait(full_a + 8 * i, last & 1, DS_WAIT_LIMIT)) atomicAdd(timeout, 1);
      }
    return;
  }

  // consumers: thread (xs, p) = (row xs of each stage, right-hand sides 2p and 2p+1)
  const int xs = tid / np, p = tid % np, r0 = 2 * p;
  const bool on0 = active[r0] != 0, on1 = active[r0 + 1] != 0;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  int64_t st = 0;
  // A wait that runs out (or `stop` set by another warp) marks the warp failed: it computes
  // nothing more but keeps the loop and barrier sequence of the others, whose waits then
  // return at once, so the block still reaches its end.
  bool failed = false;
  for (int k0 = 0; k0 < nvec; k0 += DS_VG) {
    const int nk = min(DS_VG, nvec - k0);
    df::Acc acc[DS_VG][4];  // re0, im0, re1, im1 per vector
    auto load_w = [&](int64_t x, float4& a, float4& b) {
      const bool row = x + xs < x1;
      a = (row && on0) ? w[(x + xs) * nrhs + r0] : zero;
      b = (row && on1) ? w[(x + xs) * nrhs + r0 + 1] : zero;
    };
    float4 c0, c1, n0, n1;
    load_w(x0, n0, n1);
    for (int64_t x = x0; x < x1; x += xsn, ++st) {
      c0 = n0;
      c1 = n1;
      if (x + xsn < x1) load_w(x + xsn, n0, n1);
      const int slot = (int)(st % DS_STAGES), use = (int)(st / DS_STAGES);
      if (!failed) {
        const bool landed = tc::mbar_wait_flag(full_a + 8 * slot, use & 1, DS_WAIT_LIMIT, &stop);
        if (!__all_sync(0xffffffffu, landed)) {
          failed = true;
          if (lane == 0) {
            atomicAdd(timeout, 1);
            stop = 1;
          }
        }
      }
      if (failed) continue;
      const float4* ht = reinterpret_cast<const float4*>(ds_smem + (size_t)slot * DS_STAGE_BYTES) + tid;
      const float4* lt = ht + DS_VG * (DS_TILE / 16);
      if (x + xs < x1) {
        float4 h[DS_VG], l[DS_VG];
#pragma unroll
        for (int v = 0; v < DS_VG; ++v) {
          h[v] = v < nk ? ht[v * (DS_TILE / 16)] : zero;
          l[v] = v < nk ? lt[v * (DS_TILE / 16)] : zero;
        }
#pragma unroll
        for (int v = 0; v < DS_VG; ++v) {
          // conj(a) c = (a.re c.re + a.im c.im) + i (a.re c.im - a.im c.re); a = V entry
          const float4 a0 = make_float4(h[v].x, h[v].y, l[v].x, l[v].y);
          const float4 a1 = make_float4(h[v].z, h[v].w, l[v].z, l[v].w);
          df::add_prod2(acc[v][0], a0.x, a0.z, c0.x, c0.z);
          df::add_prod2(acc[v][0], a0.y, a0.w, c0.y, c0.w);
          df::add_prod2(acc[v][1], a0.x, a0.z, c0.y, c0.w);
          df::add_prod2(acc[v][1], -a0.y, -a0.w, c0.x, c0.z);
          df::add_prod2(acc[v][2], a1.x, a1.z, c1.x, c1.z);
          df::add_prod2(acc[v][2], a1.y, a1.w, c1.y, c1.w);
          df::add_prod2(acc[v][3], a1.x, a1.z, c1.y, c1.w);
          df::add_prod2(acc[v][3], -a1.y, -a1.w, c1.x, c1.z);
        }
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(empty_a + 8 * slot);
    }
    // fold the row lanes of each warp (lane = xs_in_warp * np + p), then the warps in order
#pragma unroll
    for (int v = 0; v < DS_VG; ++v) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        for (int o = np; o < 32; o <<= 1) fold_lanes(acc[v][q], o);
      if (lane < np)
        red[warp][v][p][0] = make_double2(df::to_double(acc[v][0]), df::to_double(acc[v][1])),
        red[warp][v][p][1] = make_double2(df::to_double(acc[v][2]), df::to_double(acc[v][3]));
    }
    bar_consumers();
    for (int t = tid; t < nk * nrhs; t += DS_CONSUMERS) {
      const int v = t / nrhs, r = t % nrhs;
      double sx = 0.0, sy = 0.0;
      for (int wq = 0; wq < DS_CONSUMERS / 32; ++wq) {
        const double2 m = red[wq][v][r / 2][r & 1];
        sx += m.x;
        sy += m.y;
      }
      hpart[((int64_t)blockIdx.x * nvec + k0 + v) * nrhs + r] = make_double2(sx, sy);
    }
    bar_consumers();
  }
}

// hs[i][r] = h[i][r] as a complex double-float
__global__ void k_split_h(int count, const double2* h, float4* hs) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) hs[t] = df::split_c(h[t]);
}

// w[x][r] -= sum_{i < nvec} V_i[x][r] h_i[r]; npart[blk][r] = sum over the block of |w|^2
template <int RP>
__global__ void __launch_bounds__(256) k_orth_update_df(int64_t n, int nrhs, int nvec, const float2* __restrict__ Vh,
                                                        const float2* __restrict__ Vl, const float4* __restrict__ hs,
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
        const float2 ah = Vh[(int64_t)i * nv + x * nrhs + r], al = Vl[(int64_t)i * nv + x * nrhs + r];
        const float4 a = make_float4(ah.x, ah.y, al.x, al.y);
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

// Paired form of k_orth_update_df for an even number of right-hand sides: a lane updates
// the pair (r, r+1) of a row, reading each plane with one 16-byte load per basis vector.
template <int RP>
__global__ void __launch_bounds__(256, 4) k_orth_update_df2(int64_t n, int nrhs, int nvec, const float2* __restrict__ Vh,
                                                         const float2* __restrict__ Vl, const float4* __restrict__ hs,
                                                         const int32_t* __restrict__ active, float4* __restrict__ w,
                                                         double* __restrict__ npart) {
  constexpr int RP2 = RP / 2;
  constexpr int XL = 32 / RP2;
  __shared__ double sh[8][RP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rp = lane % RP2, xl = lane / RP2;
  const int r0 = 2 * rp;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
  const int64_t nv = n * nrhs;
  const bool in = r0 < nrhs;
  const bool on0 = in && active[min(r0, nrhs - 1)], on1 = in && active[min(r0 + 1, nrhs - 1)];
  df::Acc nrm0, nrm1;
  if (on0 || on1)
    for (int64_t x = x0 + warp * XL + xl; x < x1; x += 8 * XL) {
      df::Acc sre0, sim0, sre1, sim1;
      const int64_t q = (x * nrhs + r0) >> 1;
#pragma unroll 4
      for (int i = 0; i < nvec; ++i) {
        const float4 h = reinterpret_cast<const float4*>(Vh + (int64_t)i * nv)[q];
        const float4 l = reinterpret_cast<const float4*>(Vl + (int64_t)i * nv)[q];
        const float4 c0 = hs[i * nrhs + r0], c1 = hs[i * nrhs + r0 + 1];
        // a c = (a.re c.re - a.im c.im) + i (a.re c.im + a.im c.re)
        df::add_prod2(sre0, h.x, l.x, c0.x, c0.z);
        df::add_prod2(sre0, -h.y, -l.y, c0.y, c0.w);
        df::add_prod2(sim0, h.x, l.x, c0.y, c0.w);
        df::add_prod2(sim0, h.y, l.y, c0.x, c0.z);
        df::add_prod2(sre1, h.z, l.z, c1.x, c1.z);
        df::add_prod2(sre1, -h.w, -l.w, c1.y, c1.w);
        df::add_prod2(sim1, h.z, l.z, c1.y, c1.w);
        df::add_prod2(sim1, h.w, l.w, c1.x, c1.z);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (!(k ? on1 : on0)) continue;
        const float4 wv = w[x * nrhs + r0 + k];
        const float2 s1 = df::value(k ? sre1 : sre0), s2 = df::value(k ? sim1 : sim0);
        const float2 u = df::sub(wv.x, wv.z, s1.x, s1.y), v = df::sub(wv.y, wv.w, s2.x, s2.y);
        w[x * nrhs + r0 + k] = make_float4(u.x, v.x, u.y, v.y);
        df::Acc& nrm = k ? nrm1 : nrm0;
        df::add_prod2(nrm, u.x, u.y, u.x, u.y);
        df::add_prod2(nrm, v.x, v.y, v.x, v.y);
      }
    }
  double nd0 = df::to_double(nrm0), nd1 = df::to_double(nrm1);
#pragma unroll
  for (int o = RP2; o < 32; o <<= 1) {
    nd0 += __shfl_xor_sync(0xffffffffu, nd0, o);
    nd1 += __shfl_xor_sync(0xffffffffu, nd1, o);
  }
  if (xl == 0 && in) {
    sh[warp][r0] = nd0;
    sh[warp][r0 + 1] = nd1;
  }
  __syncthreads();
  if (threadIdx.x < RP && threadIdx.x < nrhs) {
    double s = 0;
    for (int wq = 0; wq < 8; ++wq) s += sh[wq][threadIdx.x];
    npart[(int64_t)blockIdx.x * nrhs + threadIdx.x] = s;
  }
}

// v_{j+1} = w / h_{j+1,j} into the planes (vh, vl)
__global__ void k_normalize_df(int64_t nv, int nrhs, int j, int m, const double2* H, const int32_t* active,
                               const float4* w, float2* vh, float2* vl) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const double hn = H[((int64_t)j * (m + 1) + j + 1) * nrhs + r].x;
    const float2 inv = df::split((hn > 0 && active[r]) ? 1.0 / hn : 0.0);
    const float4 a = w[t];
    const float2 u = df::mul(a.x, a.z, inv.x, inv.y), v = df::mul(a.y, a.w, inv.x, inv.y);
    vh[t] = make_float2(u.x, v.x);
    vl[t] = make_float2(u.y, v.y);
  }
}

// v0 = r / beta (r FP64) into the planes (vh, vl)
__global__ void k_scale_v0_df(int64_t nv, int nrhs, const double* beta, const int32_t* active, const double2* r,
                              float2* vh, float2* vl) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % nrhs);
    const double inv = (active[q] && beta[q] > 0) ? 1.0 / beta[q] : 0.0;
    const float4 v = df::split_c(make_double2(r[t].x * inv, r[t].y * inv));
    vh[t] = make_float2(v.x, v.y);
    vl[t] = make_float2(v.z, v.w);
  }
}

// hpart[blk][i][r] = sum over the block's rows of conj(Vh_i[x][r]) wh[x][r] with FP32
// products and sums over a lane's DOTS_U rows, FP64 from the lane reduction on (the first
// Gram-Schmidt pass). Same row split and lane layout as k_dots_df; per-warp FP64
// accumulators in shared memory.
template <int RP>
__global__ void __launch_bounds__(256) k_dots_c64(int64_t n, int nrhs, int nvec, const float2* __restrict__ Vh,
                                                  const float4* __restrict__ w, const int32_t* __restrict__ active,
                                                  double2* __restrict__ hpart) {
  constexpr int XL = 32 / RP;
  extern __shared__ double2 acc_c[];  // [8 warps][DOTS_IC][RP]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane % RP, xl = lane / RP;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = blockIdx.x * chunk, x1 = min(n, x0 + chunk);
  const int64_t nv = n * nrhs;
  const bool on = r < nrhs && active[min(r, nrhs - 1)];
  double2* my = acc_c + (size_t)warp * DOTS_IC * RP;
  for (int ic = 0; ic < nvec; ic += DOTS_IC) {
    const int icn = min(DOTS_IC, nvec - ic);
    for (int t = lane; t < DOTS_IC * RP; t += 32) my[t] = make_double2(0.0, 0.0);
    __syncwarp();
    for (int64_t xb = x0 + warp * XL; xb < x1; xb += (int64_t)8 * XL * DOTS_U) {
      float2 c[DOTS_U];
#pragma unroll
      for (int u = 0; u < DOTS_U; ++u) {
        const int64_t x = xb + (int64_t)u * 8 * XL + xl;
        if (on && x < x1) {
          const float4 wv = w[x * nrhs + r];
          c[u] = make_float2(wv.x, wv.y);
        } else {
          c[u] = make_float2(0.f, 0.f);
        }
      }
      for (int k = 0; k < icn; ++k) {
        const float2* Hi = Vh + (int64_t)(ic + k) * nv;
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int u = 0; u < DOTS_U; ++u) {
          const int64_t x = xb + (int64_t)u * 8 * XL + xl;
          const float2 a = (on && x < x1) ? Hi[x * nrhs + r] : make_float2(0.f, 0.f);
          sr = fmaf(a.x, c[u].x, fmaf(a.y, c[u].y, sr));
          si = fmaf(a.x, c[u].y, fmaf(-a.y, c[u].x, si));
        }
        double dr = sr, di = si;
#pragma unroll
        for (int o = RP; o < 32; o <<= 1) {
          dr += __shfl_xor_sync(0xffffffffu, dr, o);
          di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        if (xl == 0) {
          double2 m = my[k * RP + r];
          m.x += dr;
          m.y += di;
          my[k * RP + r] = m;
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < icn * RP; t += blockDim.x) {
      const int k = t / RP, rr = t % RP;
      double sx = 0, sy = 0;
      for (int wq = 0; wq < 8; ++wq) {
        const double2 m = acc_c[((size_t)wq * DOTS_IC + k) * RP + rr];
        sx += m.x;
        sy += m.y;
      }
      if (rr < nrhs) hpart[((int64_t)blockIdx.x * nvec + ic + k) * nrhs + rr] = make_double2(sx, sy);
    }
    __syncthreads();
  }
}

// v_{j+1}[t] = (w'[t] - sum_{i < nvec} Vh_i[t] g_i[r]) inv[r] into the planes (vh, vl): g the
// c64 rounding of the pass-2 coefficients, inv = 1 / ||w''|| as a double-float (0 for a
// finished right-hand side or a zero norm)
__global__ void __launch_bounds__(256) k_update2_normalize(int64_t nv, int nrhs, int nvec,
                                                           const float2* __restrict__ Vh,
                                                           const float2* __restrict__ g, const float2* __restrict__ inv,
                                                           const float4* __restrict__ w, float2* __restrict__ vh,
                                                           float2* __restrict__ vl) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    float cr = 0.f, ci = 0.f;
#pragma unroll 8
    for (int i = 0; i < nvec; ++i) {
      const float2 a = Vh[(int64_t)i * nv + t], b = g[i * nrhs + r];
      cr = fmaf(a.x, b.x, fmaf(-a.y, b.y, cr));
      ci = fmaf(a.x, b.y, fmaf(a.y, b.x, ci));
    }
    const float4 a = w[t];
    const float2 s = inv[r];
    const float2 u = df::sub(a.x, a.z, cr, 0.f), v = df::sub(a.y, a.w, ci, 0.f);
    const float2 ur = df::mul(u.x, u.y, s.x, s.y), vr = df::mul(v.x, v.y, s.x, s.y);
    vh[t] = make_float2(ur.x, vr.x);
    vl[t] = make_float2(ur.y, vr.y);
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

// c128 -> c64 (round to nearest) and complex double-float -> c128 (hi + lo), for mx_spmv_mixed
__global__ void k_c128_round_c64(int64_t count, const double2* __restrict__ a, float2* __restrict__ b) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    b[t] = make_float2(__double2float_rn(a[t].x), __double2float_rn(a[t].y));
}
__global__ void k_df_to_c128(int64_t count, const float4* __restrict__ w, double2* __restrict__ y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = w[t];
    y[t] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
}
void c128_to_c64(const double2* a, float2* b, int64_t count, cudaStream_t s) {
  MX_LAUNCH(k_c128_round_c64<<<grid_for(count, 256), 256, 0, s>>>(count, a, b));
  MX_CHECK_LAUNCH();
}
void df_to_c128(const float4* w, double2* y, int64_t count, cudaStream_t s) {
  MX_LAUNCH(k_df_to_c128<<<grid_for(count, 256), 256, 0, s>>>(count, w, y));
  MX_CHECK_LAUNCH();
}

// ---- host launchers ----------------------------------------------------------------------
void spmv_df(Problem& P, const float2* z, float4* w, int nrhs, cudaStream_t s) {
  const float4* coef = coef_df(P, P.xi_prob, 0, s);
  const int64_t work = P.A.rows * nrhs;
  // coefficients (16 B) and column indices once, z (c64) once, w (16 B) once
  ProfScope ps(K_SPMV, s, 1, 20.0 * P.A.nnz + 4.0 * (P.A.rows + 1) + 24.0 * (double)P.A.rows * nrhs,
               8.0 * (double)P.A.nnz * nrhs);
  if (nrhs % 2 == 0)
    MX_LAUNCH(k_spmv_df2<<<grid_for(work / 2, 256, 152LL * 32), 256, 0, s>>>(
        P.A.rows, nrhs, P.A.rowptr.p, P.A.col.p, coef, reinterpret_cast<const float4*>(z), w));
  else
    MX_LAUNCH(k_spmv_df<<<grid_for(work, 256, 152LL * 32), 256, 0, s>>>(P.A.rows, nrhs, P.A.rowptr.p, P.A.col.p,
                                                                        coef, z, w));
  MX_CHECK_LAUNCH();
}

template <int RP>
static void dots_rp(int nblk, int64_t n, int nrhs, int nvec, int with_norm, const float2* Vh, const float2* Vl,
                    const float4* w, const int32_t* active, double2* hpart, cudaStream_t s, const float4* extra) {
  const size_t smem = (size_t)8 * DOTS_IC * RP * sizeof(float4);
  static std::atomic<bool> configured{false};
  if (!configured) {
    MX_CUDA(cudaFuncSetAttribute(k_dots_df<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  if constexpr (RP >= 2) {
    if (nrhs % 2 == 0) {
      static std::atomic<bool> configured2{false};
      if (!configured2) {
        MX_CUDA(cudaFuncSetAttribute(k_dots_df2<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured2 = true;
      }
      MX_LAUNCH(k_dots_df2<RP><<<nblk, 256, smem, s>>>(n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, extra));
      return;
    }
  }
  MX_LAUNCH(k_dots_df<RP><<<nblk, 256, smem, s>>>(n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, extra));
}
int dots_df(int nblk, int64_t n, int nrhs, int nvec, int with_norm, const float2* Vh, const float2* Vl,
            const float4* w, const int32_t* active, double2* hpart, cudaStream_t s, const float4* extra,
            int32_t* timeout) {
  ProfScope ps(K_DOTS, s, 1, 16.0 * (nvec + 1) * (double)n * nrhs, 8.0 * (nvec + with_norm) * (double)n * nrhs);
  if (timeout && !extra && !with_norm && (nrhs == 2 || nrhs == 4 || nrhs == 8 || nrhs == 16 || nrhs == 32)) {
    const size_t smem = (size_t)DS_STAGES * DS_STAGE_BYTES;
    static std::atomic<bool> configured{false};
    if (!configured) {
      MX_CUDA(cudaFuncSetAttribute(k_dots_df_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      configured = true;
    }
    const int nb = std::min(nblk, 2 * sm_count());
    MX_LAUNCH(k_dots_df_staged<<<nb, DS_THREADS, smem, s>>>(n, nrhs, nvec, Vh, Vl, w, active, hpart, timeout));
    MX_CHECK_LAUNCH();
    return nb;
  }
  if (nrhs <= 1) dots_rp<1>(nblk, n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, s, extra);
  else if (nrhs <= 2) dots_rp<2>(nblk, n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, s, extra);
  else if (nrhs <= 4) dots_rp<4>(nblk, n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, s, extra);
  else if (nrhs <= 8) dots_rp<8>(nblk, n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, s, extra);
  else if (nrhs <= 16) dots_rp<16>(nblk, n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, s, extra);
  else dots_rp<32>(nblk, n, nrhs, nvec, with_norm, Vh, Vl, w, active, hpart, s, extra);
  MX_CHECK_LAUNCH();
  return nblk;
}

template <int RP>
static void dots_c64_rp(int nblk, int64_t n, int nrhs, int nvec, const float2* Vh, const float4* w,
                        const int32_t* active, double2* hpart, cudaStream_t s) {
  const size_t smem = (size_t)8 * DOTS_IC * RP * sizeof(double2);
  static std::atomic<bool> configured{false};
  if (!configured) {
    MX_CUDA(cudaFuncSetAttribute(k_dots_c64<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  MX_LAUNCH(k_dots_c64<RP><<<nblk, 256, smem, s>>>(n, nrhs, nvec, Vh, w, active, hpart));
}
void dots_c64(int nblk, int64_t n, int nrhs, int nvec, const float2* Vh, const float4* w, const int32_t* active,
              double2* hpart, cudaStream_t s) {
  // Vh (8 B per entry) once per basis vector, w once
  ProfScope ps(K_DOTS_C64, s, 1, (8.0 * nvec + 16.0) * (double)n * nrhs, 8.0 * nvec * (double)n * nrhs);
  if (nrhs <= 1) dots_c64_rp<1>(nblk, n, nrhs, nvec, Vh, w, active, hpart, s);
  else if (nrhs <= 2) dots_c64_rp<2>(nblk, n, nrhs, nvec, Vh, w, active, hpart, s);
  else if (nrhs <= 4) dots_c64_rp<4>(nblk, n, nrhs, nvec, Vh, w, active, hpart, s);
  else if (nrhs <= 8) dots_c64_rp<8>(nblk, n, nrhs, nvec, Vh, w, active, hpart, s);
  else if (nrhs <= 16) dots_c64_rp<16>(nblk, n, nrhs, nvec, Vh, w, active, hpart, s);
  else dots_c64_rp<32>(nblk, n, nrhs, nvec, Vh, w, active, hpart, s);
  MX_CHECK_LAUNCH();
}

// Paired form of k_update2_normalize (nrhs even): a thread takes the adjacent entries
// (t, t + 1) of one row, so every plane access is one 16-byte load or store.
__global__ void __launch_bounds__(256) k_update2_normalize2(int64_t nv, int nrhs, int nvec,
                                                            const float2* __restrict__ Vh,
                                                            const float2* __restrict__ g,
                                                            const float2* __restrict__ inv,
                                                            const float4* __restrict__ w, float2* __restrict__ vh,
                                                            float2* __restrict__ vl) {
  const int64_t np = nv >> 1;
  for (int64_t tp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tp < np; tp += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = tp << 1;
    const int r = (int)(t % nrhs);
    float cr0 = 0.f, ci0 = 0.f, cr1 = 0.f, ci1 = 0.f;
#pragma unroll 8
    for (int i = 0; i < nvec; ++i) {
      const float4 a = reinterpret_cast<const float4*>(Vh + (int64_t)i * nv)[tp];
      const float4 b = *reinterpret_cast<const float4*>(g + i * nrhs + r);
      cr0 = fmaf(a.x, b.x, fmaf(-a.y, b.y, cr0));
      ci0 = fmaf(a.x, b.y, fmaf(a.y, b.x, ci0));
      cr1 = fmaf(a.z, b.z, fmaf(-a.w, b.w, cr1));
      ci1 = fmaf(a.z, b.w, fmaf(a.w, b.z, ci1));
    }
    float4 oh, ol;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float4 a = w[t + k];
      const float2 sc = inv[r + k];
      const float2 u = df::sub(a.x, a.z, k ? cr1 : cr0, 0.f), v = df::sub(a.y, a.w, k ? ci1 : ci0, 0.f);
      const float2 ur = df::mul(u.x, u.y, sc.x, sc.y), vr = df::mul(v.x, v.y, sc.x, sc.y);
      if (k == 0) {
        oh.x = ur.x; oh.y = vr.x; ol.x = ur.y; ol.y = vr.y;
      } else {
        oh.z = ur.x; oh.w = vr.x; ol.z = ur.y; ol.w = vr.y;
      }
    }
    reinterpret_cast<float4*>(vh)[tp] = oh;
    reinterpret_cast<float4*>(vl)[tp] = ol;
  }
}

void update2_normalize(int64_t nv, int nrhs, int nvec, const float2* Vh, const float2* g, const float2* inv,
                       const float4* w, float2* vh, float2* vl, cudaStream_t s) {
  // Vh once per basis vector, w' once, v_{j+1} (both planes) written once
  ProfScope ps(K_ORTH_UPDATE, s, 1, (8.0 * nvec + 32.0) * (double)nv, 8.0 * nvec * (double)nv);
  if (nrhs % 2 == 0)
    MX_LAUNCH(k_update2_normalize2<<<grid_for(nv / 2, 256, 152LL * 16), 256, 0, s>>>(nv, nrhs, nvec, Vh, g, inv, w,
                                                                                     vh, vl));
  else
    MX_LAUNCH(k_update2_normalize<<<grid_for(nv, 256, 152LL * 16), 256, 0, s>>>(nv, nrhs, nvec, Vh, g, inv, w, vh, vl));
  MX_CHECK_LAUNCH();
}

template <int RP>
static void update_rp(int nblk, int64_t n, int nrhs, int nvec, const float2* Vh, const float2* Vl, const float4* hs,
                      const int32_t* active, float4* w, double* npart, cudaStream_t s) {
  if constexpr (RP >= 2) {
    if (nrhs % 2 == 0) {
      MX_LAUNCH(k_orth_update_df2<RP><<<nblk, 256, 0, s>>>(n, nrhs, nvec, Vh, Vl, hs, active, w, npart));
      return;
    }
  }
  MX_LAUNCH(k_orth_update_df<RP><<<nblk, 256, 0, s>>>(n, nrhs, nvec, Vh, Vl, hs, active, w, npart));
}
void orth_update_df(int nblk, int64_t n, int nrhs, int nvec, const float2* Vh, const float2* Vl, const double2* h,
                    float4* hs, const int32_t* active, float4* w, double* npart, cudaStream_t s) {
  {
    ProfScope ps(K_ARNOLDI_SMALL, s);
    MX_LAUNCH(k_split_h<<<grid_for((int64_t)nvec * nrhs, 128), 128, 0, s>>>(nvec * nrhs, h, hs));
    MX_CHECK_LAUNCH();
  }
  ProfScope ps(K_ORTH_UPDATE, s, 1, 16.0 * (nvec + 2) * (double)n * nrhs, 8.0 * (nvec + 0.25) * (double)n * nrhs);
  if (nrhs <= 1) update_rp<1>(nblk, n, nrhs, nvec, Vh, Vl, hs, active, w, npart, s);
  else if (nrhs <= 2) update_rp<2>(nblk, n, nrhs, nvec, Vh, Vl, hs, active, w, npart, s);
  else if (nrhs <= 4) update_rp<4>(nblk, n, nrhs, nvec, Vh, Vl, hs, active, w, npart, s);
  else if (nrhs <= 8) update_rp<8>(nblk, n, nrhs, nvec, Vh, Vl, hs, active, w, npart, s);
  else if (nrhs <= 16) update_rp<16>(nblk, n, nrhs, nvec, Vh, Vl, hs, active, w, npart, s);
  else update_rp<32>(nblk, n, nrhs, nvec, Vh, Vl, hs, active, w, npart, s);
  MX_CHECK_LAUNCH();
}

// x[t] += sum_{i < kcols[r]} z_i[t] y_i[r] (mixed form): z c64, y as double-float pairs (ys), the
// sum in double-float, added to the FP64 x once -- FP32 units instead of four FP64 FMAs per term
__global__ void __launch_bounds__(256) k_update_x_df(int64_t nv, int nrhs, const int32_t* __restrict__ kcols,
                                                     const float2* __restrict__ Z, const float4* __restrict__ ys,
                                                     double2* __restrict__ x) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t % nrhs);
    const int k = kcols[r];
    if (k == 0) continue;
    df::Acc re, im;
#pragma unroll 4
    for (int i = 0; i < k; ++i) {
      const float2 z = Z[(int64_t)i * nv + t];
      const float4 c = ys[i * nrhs + r];  // {re_hi, im_hi, re_lo, im_lo}
      df::add_prod(re, c.x, c.z, z.x);
      df::add_prod(re, -c.y, -c.w, z.y);
      df::add_prod(im, c.y, c.w, z.x);
      df::add_prod(im, c.x, c.z, z.y);
    }
    const double2 a = x[t];
    x[t] = make_double2(a.x + df::to_double(re), a.y + df::to_double(im));
  }
}

void update_x_df(int64_t nv, int nrhs, int kmax, const int32_t* kcols, const float2* Z, const double2* y, float4* ys,
                 double2* x, cudaStream_t s) {
  if (kmax <= 0) return;
  MX_LAUNCH(k_split_h<<<grid_for((int64_t)kmax * nrhs, 128), 128, 0, s>>>(kmax * nrhs, y, ys));
  MX_CHECK_LAUNCH();
  MX_LAUNCH(k_update_x_df<<<grid_for(nv, 256, 152LL * 16), 256, 0, s>>>(nv, nrhs, kcols, Z, ys, x));
  MX_CHECK_LAUNCH();
}

void normalize_df(int64_t nv, int nrhs, int j, int m, const double2* H, const int32_t* active, const float4* w,
                  float2* vh, float2* vl, cudaStream_t s) {
  ProfScope ps(K_ARNOLDI_SMALL, s, 1, 32.0 * (double)nv, 2.0 * (double)nv);
  MX_LAUNCH(k_normalize_df<<<grid_for(nv, 256), 256, 0, s>>>(nv, nrhs, j, m, H, active, w, vh, vl));
  MX_CHECK_LAUNCH();
}

void scale_v0_df(int64_t nv, int nrhs, const double* beta, const int32_t* active, const double2* r, float2* vh,
                 float2* vl, cudaStream_t s) {
  MX_LAUNCH(k_scale_v0_df<<<grid_for(nv, 256), 256, 0, s>>>(nv, nrhs, beta, active, r, vh, vl));
  MX_CHECK_LAUNCH();
}

}  // namespace mx

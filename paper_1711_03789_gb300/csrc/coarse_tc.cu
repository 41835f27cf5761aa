// Coarse apply of the mixed form with the explicit inverse on the tensor cores: Z = X R, X the
// c64 inverse of A^0 (n_c x n_c, row-major), R the restricted right-hand sides (n_c x nrhs, c64).
// The complex product is one real product: row i of X read as 2 n_c reals (re, im interleaved)
// is the K-major A operand as it lies in memory, and the right-hand sides of a group of 16 form
// the 32 rows of the K-major B operand,
//   B[c][2j] = Re r_jc, B[c][2j+1] = -Im r_jc          (columns c < 16: Re z_ic)
//   B[16+c][2j] = Im r_jc, B[16+c][2j+1] = Re r_jc     (columns 16 + c: Im z_ic),
// so D = A B^T holds Re Z and Im Z side by side. Every FP32 value enters as a TF32 pair
// (hi rounded to nearest, lo the exact remainder) and three products are kept per term
// (hi*hi + hi*lo + lo*hi, about 1.2e-6 relative error each), accumulated in FP32 in TMEM.
//
// A CTA owns 128 rows of X (the TMEM lanes) and a range of its columns (split-K over
// blockIdx.y, so that the grid is about one wave of two CTAs per SM); X leaves HBM once. Per
// chunk of 16 complex columns its 256 threads load 16 KB of X (one 16-byte load per core-matrix
// row, two chunks ahead in registers), split them into TF32 planes in shared memory and one
// thread issues the 12 MMAs; the partial products go to part[ks][i][r] and k_coarse_sum adds
// the splits in a fixed order.
#include "problem.cuh"
#include "tc.cuh"

namespace mx {

namespace {

constexpr int CT_M = 128;                        // rows of X per CTA (TMEM lanes)
constexpr int CT_KC = 16;                        // complex columns per chunk: 32 real K
constexpr int CT_G = 16;                         // right-hand sides per group (N = 32)
constexpr int CT_THREADS = 256;
constexpr uint32_t CT_LBO = 128;                 // K-adjacent core matrices
constexpr uint32_t CT_SBO = 1024;                // 8-row groups: 8 core matrices of K = 4
constexpr int CT_APLANE = CT_M * 32 * 4;         // one TF32 plane of the X tile: 16 KB
constexpr int CT_BPLANE = 2 * CT_G * 32 * 4;     // one TF32 plane of the right-hand-side tile: 4 KB
constexpr int CT_STAGE = 2 * CT_APLANE + 2 * CT_BPLANE;
constexpr int CT_SMEM = 2 * CT_STAGE;            // two stages: 80 KB
constexpr int CT_WAIT = 1 << 22;

// 32 real K values of one operand row: D (+)= A_plane * B_plane^T (four K = 8 instructions)
__device__ __forceinline__ void gemm_k32(uint32_t d, uint32_t a, uint32_t b, uint32_t id, bool first) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    tc::mma_tf32(d, tc::sdesc(a + kk * 256, CT_LBO, CT_SBO), tc::sdesc(b + kk * 256, CT_LBO, CT_SBO), id,
                 (first && kk == 0) ? 0u : 1u);
}

__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t o, float4 v) {
  const float4 h = make_float4(tc::tf32_rn(v.x), tc::tf32_rn(v.y), tc::tf32_rn(v.z), tc::tf32_rn(v.w));
  *reinterpret_cast<float4*>(hi + o) = h;
  *reinterpret_cast<float4*>(lo + o) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

struct Chunk {
  float4 x[4];  // four consecutive core-matrix rows (K groups) of one row of the X tile
  float4 b;     // one core-matrix row of the right-hand-side tile
};

}  // namespace

__global__ void __launch_bounds__(CT_THREADS, 2) k_coarse_dense_tc(int n, int nrhs, int kspan, const float2* __restrict__ X,
                                                                   const float2* __restrict__ rc,
                                                                   float2* __restrict__ part, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char ct_smem[];
  __shared__ __align__(8) uint64_t mb[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * CT_M, ks = blockIdx.y, g0 = blockIdx.z * CT_G;
  const int gn = min(CT_G, nrhs - g0);
  const int jbeg = ks * kspan, jend = min(n, jbeg + kspan);
  const int nch = jend > jbeg ? (jend - jbeg + CT_KC - 1) / CT_KC : 0;
  const uint32_t mb_a = tc::smem_u32(&mb[0]);
  if (tid == 0) {
    tc::mbar_init(mb_a, 1);
    tc::mbar_init(mb_a + 8, 1);
    tc::mbar_fence_init();
    failed_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), 32);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;

  // this thread's share of a chunk: row xr = tid % 128 of the X tile, complex columns 8 h ..
  // 8 h + 7 (h = tid / 128: four core-matrix rows, 64 contiguous bytes); row nb = tid % 32 of
  // the right-hand-side tile at complex columns 2 kb, 2 kb + 1 (kb = tid / 32). Consecutive
  // threads take consecutive rows, so the 8 threads of a 16-byte shared-memory store phase write
  // 8 different 16-byte bank groups of the no-swizzle layout (one row's K groups all share one).
  const int xr = tid & (CT_M - 1), h = tid >> 7, nb = tid & 31, kb = tid >> 5;
  auto load = [&](int c, Chunk& ch) {
    const int jc = jbeg + c * CT_KC;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = jc + 8 * h + 2 * q;  // jend even: a pair is wholly in or out
      ch.x[q] = (j < jend && i0 + xr < n) ? *reinterpret_cast<const float4*>(X + (int64_t)(i0 + xr) * n + j)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int j = jc + 2 * kb, cc = nb & (CT_G - 1);
    float2 r0 = make_float2(0.f, 0.f), r1 = r0;
    if (j < jend && cc < gn) {
      r0 = rc[(int64_t)j * nrhs + g0 + cc];
      r1 = rc[(int64_t)(j + 1) * nrhs + g0 + cc];
    }
    ch.b = nb < CT_G ? make_float4(r0.x, -r0.y, r1.x, -r1.y) : make_float4(r0.y, r0.x, r1.y, r1.x);
  };
  auto stage = [&](int c, const Chunk& ch) {
    unsigned char* s = ct_smem + (c & 1) * CT_STAGE;
#pragma unroll
    for (int q = 0; q < 4; ++q) put_split(s, s + CT_APLANE, tc::kmaj(xr, 4 * (4 * h + q), CT_LBO, CT_SBO), ch.x[q]);
    put_split(s + 2 * CT_APLANE, s + 2 * CT_APLANE + CT_BPLANE, tc::kmaj(nb, 4 * kb, CT_LBO, CT_SBO), ch.b);
  };
  const uint32_t idesc = tc::idesc_tf32(CT_M, 2 * CT_G);
  auto issue = [&](int c) {
    const uint32_t s = tc::smem_u32(ct_smem) + (c & 1) * CT_STAGE;
    const uint32_t ah = s, al = s + CT_APLANE, bh = s + 2 * CT_APLANE, bl = bh + CT_BPLANE;
    gemm_k32(tmem, ah, bh, idesc, c == 0);
    gemm_k32(tmem, ah, bl, idesc, false);
    gemm_k32(tmem, al, bh, idesc, false);
    tc::mma_commit(mb_a + 8 * (c & 1));
  };

  Chunk ca, cb;  // chunks c (even) and c + 1 (odd) in flight
  if (nch > 0) load(0, ca);
  if (nch > 1) load(1, cb);
  int issued = 0;  // chunks whose MMAs were issued (the same count in every thread)
  for (int c = 0; c < nch; ++c) {
    // the stage about to be written was read by the MMAs of chunk c - 2
    bool ok = true;
    if (c >= 2) ok = tc::mbar_wait(mb_a + 8 * (c & 1), ((c - 2) >> 1) & 1, CT_WAIT);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicAdd(status + 2, 1);
        failed_s = 1;
      }
      break;
    }
    if (c & 1) {
      stage(c, cb);
      if (c + 2 < nch) load(c + 2, cb);
    } else {
      stage(c, ca);
      if (c + 2 < nch) load(c + 2, ca);
    }
    tc::fence_proxy_async();  // the planes written above are read by the tensor cores
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      issue(c);
    }
    issued = c + 1;
  }
  // the last commit covers every MMA the CTA issued (after a failure too: nothing is left
  // running when the TMEM is read or freed)
  if (issued > 0) {
    const int c = issued - 1;
    const bool ok = tc::mbar_wait(mb_a + 8 * (c & 1), (c >> 1) & 1, CT_WAIT);
    if (__syncthreads_or(!ok) && tid == 0) {
      atomicAdd(status + 2, 1);
      failed_s = 1;
    }
  }
  __syncthreads();
  tc::fence_after();
  if (warp < 4) {
    const int i = i0 + 32 * warp + lane;
    uint32_t r[32];
    if (issued == nch && nch > 0 && !failed_s) {
      tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), r);
    } else {
#pragma unroll
      for (int t = 0; t < 32; ++t) r[t] = 0u;
    }
    if (i < n) {
      float2* o = part + ((int64_t)ks * n + i) * nrhs + g0;
#pragma unroll
      for (int t = 0; t < CT_G; ++t)
        if (t < gn) o[t] = make_float2(__uint_as_float(r[t]), __uint_as_float(r[CT_G + t]));
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// Z = X R as above into part (ks splits of the columns of X) and its split count; false when
// the shape does not suit the kernel (odd n_c: a pair of complex columns must start 16-byte
// aligned).
bool coarse_dense_tc(Problem& P, const float2* rin, int nrhs, float2*& part, int& ks) {
  const int64_t nc = P.n_c;
  if (nc % 2 != 0 || nc > (1 << 30) / CT_M) return false;
  cudaStream_t s = P.stream;
  static std::atomic<bool> configured{false};
  if (!configured) {
    MX_CUDA(cudaFuncSetAttribute(k_coarse_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, CT_SMEM));
    configured = true;
  }
  const int mt = (int)((nc + CT_M - 1) / CT_M);
  const int groups = (nrhs + CT_G - 1) / CT_G;
  // about one wave of two CTAs per SM; every split a whole number of chunks
  ks = std::max(1, std::min(64, (2 * sm_count()) / (mt * groups)));
  const int kspan = (int)(((nc + ks - 1) / ks + CT_KC - 1) / CT_KC) * CT_KC;
  ks = (int)((nc + kspan - 1) / kspan);
  P.c_part.ensure((size_t)ks * nc * nrhs);
  part = P.c_part.p;
  MX_LAUNCH(k_coarse_dense_tc<<<dim3(mt, ks, groups), CT_THREADS, CT_SMEM, s>>>((int)nc, nrhs, kspan, P.A0inv.p, rin,
                                                                                part, P.status.p));
  MX_CHECK_LAUNCH();
  return true;
}

}  // namespace mx

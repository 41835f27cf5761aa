// Batched band LU of the c64 local matrices (Eq. 3.3, factored for the local solves of
// Eq. 3.4) in one persistent launch: one CTA factors one subdomain matrix from its first
// to its last block column, so the trailing window it updates (b x b entries, about 1 MB
// at b = 347) stays in L2 from one step to the next instead of streaming through HBM once
// per step, as it does when every step is a separate launch over the whole batch.
//
// Step with the diagonal block [k0, k0 + kb), kb <= 32, and window W = [k1, k1 + span),
// k1 = k0 + kb, span = min(n - k1, b) (the window lies inside the band):
//   1. LU of the diagonal block in shared memory (CUDA cores, no pivoting);
//   2. panels L21 = A21 U11^{-1} (rows of W) and U12 = L11^{-1} A12 (columns of W), one
//      thread per row or column with the 32 unknowns in registers (CUDA cores);
//   3. A22 -= L21 U12 over W x W on the tensor cores (tcgen05, kind::tf32, FP32 accumulation
//      in tensor memory), tile by tile (128 rows x 128 complex columns).
// A complex tile product is four real GEMMs: Re D = Lr Ur - Li Ui, Im D = Lr Ui + Li Ur (the
// minus sign by the instruction descriptor's negate-A bit). Each operand element x enters as
// hi + lo, hi = the TF32 truncation of x and lo = x - hi, and the product as
// hi*hi + hi*lo + lo*hi (three TF32 products, close to FP32 accuracy; the lo*lo term is below
// FP32 resolution). Operands are staged by the threads from the band storage (L2) into shared
// memory in the canonical no-swizzle K-major layout, four planes per tile (re hi, im hi,
// re lo, im lo); the A tile (rows of L21) is staged once per tile row, the B tiles (columns of
// U12) into two buffers, and the accumulators use two TMEM slots, so the staging of tile q + 1
// and the epilogue of tile q - 1 (TMEM -> registers, A22 -= D in the band storage) run while
// the tensor cores work on tile q.
//
// The factors are bit-for-bit those of the same arithmetic done elsewhere only up to the
// order of the FP32 accumulation; they are the no-pivot LU of the band (no fill outside it).
// Every wait is bounded: a wait that runs out counts in status[2]; the block then stops at the
// next barrier (__syncthreads_or keeps the decision uniform), frees its tensor memory and returns.
#include "problem.cuh"
#include "tc.cuh"

namespace mx {

namespace {

constexpr int NB = LU_NB;                   // columns per step (complex K of the update)
constexpr int FT = 128;                     // tile rows (TMEM lanes) = tile complex columns
constexpr uint32_t F_LBO = 128;             // K-adjacent core matrices
constexpr uint32_t F_SBO = (NB / 4) * 128;  // 8-row groups (1024 B)
constexpr int PLANE = FT * NB * 4;          // one TF32 plane of a tile: 16 KB
constexpr int TILE = 4 * PLANE;             // re hi, im hi, re lo, im lo: 64 KB
constexpr int F_SMEM = 3 * TILE;            // A tile + two B tiles: 192 KB
constexpr int F_WAIT = 1 << 22;             // poll limit of an mbarrier wait
constexpr uint32_t NEG_A = 1u << 13;        // instruction descriptor: negate A

__device__ __forceinline__ uint32_t bits_abs(float2 v) { return __float_as_uint(sqrtf(v.x * v.x + v.y * v.y)); }

// one real GEMM of the tile: D (+)= A_plane * B_plane^T over K = 32 (four K = 8 instructions)
__device__ __forceinline__ void gemm32(uint32_t d, uint32_t a, uint32_t b, uint32_t id, bool first) {
#pragma unroll
  for (int kk = 0; kk < NB / 8; ++kk)
    tc::mma_tf32(d, tc::sdesc(a + kk * 256, F_LBO, F_SBO), tc::sdesc(b + kk * 256, F_LBO, F_SBO), id,
                 (first && kk == 0) ? 0u : 1u);
}

}  // namespace

template <int SPLIT>
__global__ void __launch_bounds__(256, 1) k_band_lu_tc(BandBatch B, float2* A, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ float2 s[NB][NB + 1];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;

  const int m = blockIdx.x;
  const int n = B.n[m], b = B.b[m], ld = B.ld[m];
  const int64_t off = B.off[m];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* aop = smem;
  const uint32_t a_s = tc::smem_u32(smem);
  const uint32_t mb[2] = {tc::smem_u32(&mbar[0]), tc::smem_u32(&mbar[1])};

  if (tid == 0) {
    tc::mbar_init(mb[0], 1);
    tc::mbar_init(mb[1], 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;

  uint32_t par[2] = {0u, 0u};  // parity of the next completion of each slot's barrier
  int my_fail = 0;
  bool failed = false;
  uint32_t um = 0;  // largest |U| entry this thread finalised (pivot growth)

  for (int k0 = 0; k0 < n && !failed; k0 += NB) {
    const int kb = min(NB, n - k0);
    const int k1 = k0 + kb;
    const int span = min(n - k1, b);

    // ---- 1. diagonal block
    for (int t = tid; t < NB * NB; t += blockDim.x) {
      const int i = t % NB, j = t / NB;
      float2 v = make_float2(0.f, 0.f);
      if (i < kb && j < kb && abs(i - j) <= b) v = A[bidx(off, ld, b, k0 + i, k0 + j)];
      s[i][j] = v;
    }
    __syncthreads();
    for (int k = 0; k < kb; ++k) {
      const float2 piv = s[k][k];
      const float p2 = cabs2(piv);
      if (tid == 0 && !(p2 > 0 && p2 < INFINITY)) atomicAdd(status, 1);
      const float2 inv = crcp(piv);
      __syncthreads();
      for (int i = k + 1 + tid; i < kb; i += blockDim.x) s[i][k] = cmul(s[i][k], inv);
      __syncthreads();
      const int w = kb - k - 1;
      for (int t = tid; t < w * w; t += blockDim.x) {
        const int i = k + 1 + t % w, j = k + 1 + t / w;
        float2 v = s[i][j];
        cfms(v, s[i][k], s[k][j]);
        s[i][j] = v;
      }
      __syncthreads();
    }
    for (int t = tid; t < kb * kb; t += blockDim.x) {
      const int i = t % kb, j = t / kb;
      if (abs(i - j) <= b) {
        A[bidx(off, ld, b, k0 + i, k0 + j)] = s[i][j];
        if (i <= j) um = max(um, bits_abs(s[i][j]));
      }
    }
    if (span <= 0) break;  // last block column (span is the same for every thread)

    // ---- 2. panels: rows [0, span) of L21, columns [span, 2 span) of U12
    for (int t = tid; t < 2 * span; t += blockDim.x) {
      float2 x[NB];
      if (t < span) {
        const int i = k1 + t;
#pragma unroll
        for (int k = 0; k < NB; ++k)
          x[k] = (k < kb && i - (k0 + k) <= b) ? A[bidx(off, ld, b, i, k0 + k)] : make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NB; ++k) {  // x U11 = a
          if (k < kb) {
            float2 v = x[k];
#pragma unroll
            for (int j = 0; j < k; ++j) cfms(v, x[j], s[j][k]);
            x[k] = cmul(v, crcp(s[k][k]));
          }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < kb && i - (k0 + k) <= b) A[bidx(off, ld, b, i, k0 + k)] = x[k];
      } else {
        const int j = k1 + t - span;
#pragma unroll
        for (int k = 0; k < NB; ++k)
          x[k] = (k < kb && j - (k0 + k) <= b) ? A[bidx(off, ld, b, k0 + k, j)] : make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NB; ++k) {  // L11 y = a (unit lower)
          if (k < kb) {
            float2 v = x[k];
#pragma unroll
            for (int j2 = 0; j2 < k; ++j2) cfms(v, s[k][j2], x[j2]);
            x[k] = v;
          }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < kb && j - (k0 + k) <= b) {
            A[bidx(off, ld, b, k0 + k, j)] = x[k];
            um = max(um, bits_abs(x[k]));
          }
      }
    }
    __syncthreads();

    // ---- 3. A22 -= L21 U12 over the window, tiles of 128 x 128 complex entries
    const int nt = (span + FT - 1) / FT;
    const int lim = k1 + span;
    // stage rows [r0, r0 + 128) of L21 (A) or columns [r0, r0 + 128) of U12 (B) into a tile
    // (the four items of a thread load first, so their 16 reads are in flight together)
    constexpr int ITEMS = FT * (NB / 4) / 256;
    auto stage = [&](unsigned char* dst, int r0, bool rows) {
      float2 v[ITEMS][4];
#pragma unroll
      for (int it2 = 0; it2 < ITEMS; ++it2) {
        const int t = tid + 256 * it2;
        const int r = t % FT, g = t / FT;
        const int e = r0 + r;  // row of L21 or column of U12
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int kc = 4 * g + u, k = k0 + kc;
          v[it2][u] = make_float2(0.f, 0.f);
          if (kc < kb && e < lim && e - k <= b)
            v[it2][u] = rows ? A[bidx(off, ld, b, e, k)] : A[bidx(off, ld, b, k, e)];
        }
      }
#pragma unroll
      for (int it2 = 0; it2 < ITEMS; ++it2) {
        const int t = tid + 256 * it2;
        const int r = t % FT, g = t / FT;
        float hr[4], hi_[4], lr[4], li[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          hr[u] = tc::tf32_hi(v[it2][u].x);
          hi_[u] = tc::tf32_hi(v[it2][u].y);
          lr[u] = v[it2][u].x - hr[u];
          li[u] = v[it2][u].y - hi_[u];
        }
        const uint32_t o = tc::kmaj(r, 4 * g, F_LBO, F_SBO);
        *reinterpret_cast<float4*>(dst + o) = make_float4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<float4*>(dst + PLANE + o) = make_float4(hi_[0], hi_[1], hi_[2], hi_[3]);
        if (SPLIT == 3) {
          *reinterpret_cast<float4*>(dst + 2 * PLANE + o) = make_float4(lr[0], lr[1], lr[2], lr[3]);
          *reinterpret_cast<float4*>(dst + 3 * PLANE + o) = make_float4(li[0], li[1], li[2], li[3]);
        }
      }
    };
    // TMEM -> registers -> A22 -= D for tile p (slot p & 1: Re D in columns [0, 128), Im D in
    // [128, 256) of the slot); returns false if the tensor cores did not finish in time
    auto epilogue = [&](int p) -> bool {
      const int sl = p & 1;
      const bool ok = tc::mbar_wait(mb[sl], par[sl], F_WAIT);
      par[sl] ^= 1u;
      tc::fence_after();
      if (!ok) return false;
      const int i0 = k1 + FT * (p / nt), j0 = k1 + FT * (p % nt);
      const int lg = warp & 3, half = warp >> 2;
      const int i = i0 + 32 * lg + lane;
      const uint32_t base = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(256 * sl);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = 64 * half + 32 * c;
        uint32_t vr[32], vi[32];
        tc::tmem_ld32(base + col, vr);
        tc::tmem_ld32(base + 128 + col, vi);
        if (i < lim) {
          // 16 entries of the row per round: all loads first, then the stores (the stores
          // could alias later loads for the compiler, which would serialise every pair)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 x[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int j = j0 + col + 16 * h + q;
              x[q] = j < lim ? A[bidx(off, ld, b, i, j)] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int j = j0 + col + 16 * h + q;
              if (j < lim) {
                x[q].x -= __uint_as_float(vr[16 * h + q]);
                x[q].y -= __uint_as_float(vi[16 * h + q]);
                A[bidx(off, ld, b, i, j)] = x[q];
              }
            }
          }
        }
      }
      return true;
    };

    int pending = -1;
    for (int q = 0; q < nt * nt; ++q) {
      const int it = q / nt, jt = q % nt, sl = q & 1;
      unsigned char* bop = smem + TILE * (1 + sl);
      if (jt == 0) {
        if (pending >= 0) {  // the A tile is about to change: its last product must be done
          if (!epilogue(pending)) my_fail = 1;
          pending = -1;
        }
        stage(aop, k1 + FT * it, true);
      }
      stage(bop, k1 + FT * jt, false);
      tc::fence_proxy_async();
      tc::fence_before();
      if (__syncthreads_or(my_fail)) {
        failed = true;
        break;
      }
      tc::fence_after();
      if (tid == 0) {
        const uint32_t idp = tc::idesc_tf32(FT, FT), idn = idp | NEG_A;
        const uint32_t b_s = tc::smem_u32(bop);
        const uint32_t dr = tmem + (uint32_t)(256 * sl), di = dr + 128;
        const uint32_t A0 = a_s, A1 = a_s + PLANE, A2 = a_s + 2 * PLANE, A3 = a_s + 3 * PLANE;
        const uint32_t B0 = b_s, B1 = b_s + PLANE, B2 = b_s + 2 * PLANE, B3 = b_s + 3 * PLANE;
        gemm32(dr, A0, B0, idp, true);   // + Lr Ur
        gemm32(dr, A1, B1, idn, false);  // - Li Ui
        gemm32(di, A0, B1, idp, true);   // + Lr Ui
        gemm32(di, A1, B0, idp, false);  // + Li Ur
        if (SPLIT == 3) {
          gemm32(dr, A0, B2, idp, false);
          gemm32(dr, A2, B0, idp, false);
          gemm32(dr, A1, B3, idn, false);
          gemm32(dr, A3, B1, idn, false);
          gemm32(di, A0, B3, idp, false);
          gemm32(di, A2, B1, idp, false);
          gemm32(di, A1, B2, idp, false);
          gemm32(di, A3, B0, idp, false);
        }
        tc::mma_commit(mb[sl]);
      }
      if (pending >= 0 && !epilogue(pending)) my_fail = 1;
      pending = q;
    }
    if (!failed && pending >= 0 && !epilogue(pending)) my_fail = 1;
    tc::fence_before();
    if (__syncthreads_or(my_fail)) failed = true;  // the window is updated before the next step reads it
    tc::fence_after();
  }

  if (failed && tid == 0) atomicAdd(status + 2, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
  if (B.umax) {
    um = __reduce_max_sync(0xffffffffu, um);
    if (lane == 0) atomicMax(B.umax + m, um);
  }
}

void band_lu_fused(const BandBatch& B, float2* A, int split, int32_t* status, cudaStream_t s, double bytes,
                   double flops) {
  static bool attr1 = false, attr3 = false;
  ProfScope ps(K_LU_UPDATE, s, 1, bytes, flops);
  if (split == 3) {
    if (!attr3) {
      MX_CUDA(cudaFuncSetAttribute(k_band_lu_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM));
      attr3 = true;
    }
    MX_LAUNCH(k_band_lu_tc<3><<<B.count, 256, F_SMEM, s>>>(B, A, status));
  } else {
    if (!attr1) {
      MX_CUDA(cudaFuncSetAttribute(k_band_lu_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM));
      attr1 = true;
    }
    MX_LAUNCH(k_band_lu_tc<1><<<B.count, 256, F_SMEM, s>>>(B, A, status));
  }
  MX_CHECK_LAUNCH();
}

}  // namespace mx

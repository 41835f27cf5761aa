// Trailing update of the batched band LU on the 5th-generation tensor cores (tcgen05).
//
// For the step with diagonal block [k0, k0 + kb), every matrix of the batch gets
// A22 -= L21 U12 over its band window (Sec. 3.3 local minors, factored for Eq. 3.4).
// One CTA computes a 128 x 64 complex output tile as a real GEMM of M = 128, N = 128,
// K = 2 kb with the complex product embedded in real arithmetic:
//   A'[i][2k + c]  = (Re, Im) of L(i, k)                         (K-major)
//   B'[2j][2k + c] = (Re, -Im) of U(k, j), B'[2j+1][2k + c] = (Im, Re) of U(k, j)
// so D[i][2j] = Re(L U)(i, j) and D[i][2j + 1] = Im(L U)(i, j). Operands are staged by
// the threads into shared memory in the canonical no-swizzle K-major layout (core
// matrices of 8 rows x 16 bytes); one elected thread issues tcgen05.mma kind::tf32 with
// the FP32 accumulator in tensor memory; the epilogue reads TMEM with tcgen05.ld and
// subtracts the tile from the band storage in place.
//
// Precision: split = 3 evaluates hi*hi + hi*lo + lo*hi with x = hi + lo, hi the TF32
// truncation of x (three TF32 products, FP32 accumulation: close to FP32 accuracy);
// split = 1 uses one TF32 product.
//
// Waits are bounded: if the MMA completion barrier does not flip within the limit the
// block records an error in status[2], skips its epilogue, frees its TMEM and returns.
#include "problem.cuh"

namespace mx {

namespace {

constexpr int TM = 128;          // tile rows (TMEM lanes)
constexpr int TNC = 64;          // tile complex columns (N = 128 real)
constexpr int TKR = 2 * LU_NB;   // real K of one step (64)
constexpr int TILE_BYTES = TM * TKR * 4;  // one operand tile: 32 KB
constexpr uint32_t LBO = 128;             // K-adjacent core matrices
constexpr uint32_t SBO = (TKR / 4) * 128; // 8-row groups

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, kreal) in the canonical K-major no-swizzle layout
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return (row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // sm_100-family descriptor version; no swizzle, base offset 0
  return d;
}

__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4)                  // D: f32
         | (2u << 7) | (2u << 10)   // A, B: tf32
         | ((uint32_t)(128 >> 3) << 17)  // N = 128
         | ((uint32_t)(TM >> 4) << 24);  // M = 128
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc_tf32()), "r"(acc));
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

}  // namespace

template <int SPLIT>
__global__ void __launch_bounds__(256, 1) k_lu_update_tc(BandBatch B, float2* A, int k0, int tiles_r, int tiles_c,
                                                         int32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_hi = smem;
  unsigned char* b_hi = smem + TILE_BYTES;
  unsigned char* a_lo = smem + 2 * TILE_BYTES;
  unsigned char* b_lo = smem + 3 * TILE_BYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;

  const int m = blockIdx.x;
  const int n = B.n[m], b = B.b[m], ld = B.ld[m];
  const int64_t off = B.off[m];
  if (k0 >= n) return;
  const int kb = min(LU_NB, n - k0);
  const int k1 = k0 + kb;
  const int span = min(n, k1 + b) - k1;
  if (span <= 0) return;
  const int tr = (span + TM - 1) / TM, tc = (span + TNC - 1) / TNC;
  if ((int)blockIdx.y >= tr * tc) return;
  const int i0 = k1 + TM * ((int)blockIdx.y % tr), j0 = k1 + TNC * ((int)blockIdx.y / tr);
  if (i0 - (j0 + TNC - 1) > b || j0 - (i0 + TM - 1) > b) return;  // tile outside the band

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- stage A' = L21 tile (128 rows x kb complex) and B' = U12 tile (kb x 64 complex)
  for (int t = tid; t < TM * LU_NB; t += blockDim.x) {
    const int r = t % TM, kc = t / TM;
    const int i = i0 + r, k = k0 + kc;
    float2 v = make_float2(0.f, 0.f);
    if (kc < kb && i < n && i - k <= b) v = A[bidx(off, ld, b, i, k)];
    const uint32_t o = kmaj(r, 2 * kc);
    const float2 h = make_float2(tf32_hi(v.x), tf32_hi(v.y));
    *reinterpret_cast<float2*>(a_hi + o) = h;
    if (SPLIT == 3) *reinterpret_cast<float2*>(a_lo + o) = make_float2(v.x - h.x, v.y - h.y);
  }
  for (int t = tid; t < LU_NB * TNC; t += blockDim.x) {
    const int kc = t % LU_NB, jc = t / LU_NB;
    const int k = k0 + kc, j = j0 + jc;
    float2 u = make_float2(0.f, 0.f);
    if (kc < kb && j < n && j - k <= b) u = A[bidx(off, ld, b, k, j)];
    const uint32_t o_re = kmaj(2 * jc, 2 * kc), o_im = kmaj(2 * jc + 1, 2 * kc);
    const float2 h = make_float2(tf32_hi(u.x), tf32_hi(u.y));
    *reinterpret_cast<float2*>(b_hi + o_re) = make_float2(h.x, -h.y);
    *reinterpret_cast<float2*>(b_hi + o_im) = make_float2(h.y, h.x);
    if (SPLIT == 3) {
      const float2 l = make_float2(u.x - h.x, u.y - h.y);
      *reinterpret_cast<float2*>(b_lo + o_re) = make_float2(l.x, -l.y);
      *reinterpret_cast<float2*>(b_lo + o_im) = make_float2(l.y, l.x);
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  // ---- MMA: 8 K-steps (K = 8 tf32 each) per product
  if (tid == 0) {
    const uint32_t ah = smem_u32(a_hi), bh = smem_u32(b_hi), al = smem_u32(a_lo), bl = smem_u32(b_lo);
    uint32_t acc = 0;
    for (int kk = 0; kk < TKR / 8; ++kk) {
      mma_tf32(tmem, sdesc(ah + kk * 256), sdesc(bh + kk * 256), acc);
      acc = 1;
      if (SPLIT == 3) {
        mma_tf32(tmem, sdesc(ah + kk * 256), sdesc(bl + kk * 256), 1);
        mma_tf32(tmem, sdesc(al + kk * 256), sdesc(bh + kk * 256), 1);
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
  }
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(&mbar)), "r"(0));
  }
  if (!done && lane == 0) atomicAdd(status, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");

  // ---- epilogue: warps w and w + 4 share TMEM lanes 32 (w % 4) ..; columns split in halves
  if (done) {
    const int lg = warp & 3, half = warp >> 2;
    const int r = 32 * lg + lane, i = i0 + r;
    for (int c = 0; c < 2; ++c) {
      const int col0 = 64 * half + 32 * c;  // real column (TMEM column)
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * lg) << 16) + col0, v);
      if (i < n) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = j0 + col0 / 2 + q;
          if (j < n && abs(i - j) <= b) {
            float2* p = A + bidx(off, ld, b, i, j);
            float2 x = *p;
            x.x -= __uint_as_float(v[2 * q]);
            x.y -= __uint_as_float(v[2 * q + 1]);
            *p = x;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// host launcher (one step of the batched band LU, FP32 factors)
void lu_update_tc(const BandBatch& B, float2* A, int k0, int max_span, int split, int32_t* status, cudaStream_t s) {
  const int tr = (max_span + TM - 1) / TM, tc = (max_span + TNC - 1) / TNC;
  const int smem = (split == 3 ? 4 : 2) * TILE_BYTES;
  static std::atomic<bool> attr1{false}, attr3{false};
  if (split == 3) {
    if (!attr3) {
      MX_CUDA(cudaFuncSetAttribute(k_lu_update_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      attr3 = true;
    }
    MX_LAUNCH(k_lu_update_tc<3><<<dim3(B.count, tr * tc), 256, smem, s>>>(B, A, k0, tr, tc, status));
  } else {
    if (!attr1) {
      MX_CUDA(cudaFuncSetAttribute(k_lu_update_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      attr1 = true;
    }
    MX_LAUNCH(k_lu_update_tc<1><<<dim3(B.count, tr * tc), 256, smem, s>>>(B, A, k0, tr, tc, status));
  }
  MX_CHECK_LAUNCH();
}

}  // namespace mx

// Batched band LU of the c64 local matrices (Eq. 3.3, factored for the local solves of
// Eq. 3.4) in one persistent launch: one CTA factors one subdomain matrix from its first
// to its last block column, so the trailing window it updates (b x b entries, about 1 MB
// at b = 347) stays close (L2) from one step to the next instead of streaming through HBM
// once per step, as it does when every step is a separate launch over the whole batch.
//
// Step with the diagonal block [k0, k0 + kb), kb <= 32, and window W = [k1, k1 + span),
// k1 = k0 + kb, span = min(n - k1, b) (the window lies inside the band):
//   1. LU of the diagonal block in shared memory (CUDA cores, no pivoting), then the inverses
//      L11^{-1} and U11^{-1} by row operations in shared memory; they are written out as the
//      inverted diagonal blocks the local solves apply;
//   2. panels L21 = A21 U11^{-1} (rows of W) and U12 = L11^{-1} A12 (columns of W; computed as
//      U12^T = A12^T L11^{-T}) on the tensor cores, 128-row tiles with N = 32;
//   3. A22 -= L21 U12 over W x W on the tensor cores, tiles of 128 rows x 128 complex columns.
// Tensor-core products use tcgen05 kind::tf32 with FP32 accumulation in tensor memory. A
// complex product is four real GEMMs: Re D = Ar Br - Ai Bi, Im D = Ar Bi + Ai Br (the minus
// sign by the instruction descriptor's negate-A bit). Each operand element x enters as
// hi + lo, hi = x rounded to the nearest TF32 value and lo = x - hi (|lo| <= 2^-11 |x|, read
// by the tensor core with its low 13 bits dropped), and a product as hi*hi + hi*lo + lo*hi:
// three TF32 products with a relative error of about 2.5 * 2^-21 (1.2e-6) per product,
// against 2^-24 for an FP32 multiply-add; the accumulation is FP32.
// Operands are staged by the threads from the band storage (L2) into shared memory in the
// canonical no-swizzle K-major layout, four planes per tile (re hi, im hi, re lo, im lo).
// In the update the A tile (rows of L21) is staged once per tile row and the B tiles (columns
// of U12) into two buffers with two TMEM accumulator slots, so the staging of tile q + 1 and
// the epilogue of tile q - 1 (TMEM -> registers, A22 -= D in the band storage) run while the
// tensor cores work on tile q.
//
// The factors are the no-pivot LU of the band (no fill outside it) in FP32 arithmetic, with
// the panels formed from the inverted diagonal blocks instead of by substitution (the same
// factors up to rounding). Every wait is bounded: a wait that runs out counts in status[2];
// the block then stops at the next barrier (__syncthreads_or keeps the decision uniform),
// frees its tensor memory and returns.
#include "problem.cuh"
#include "tc.cuh"

namespace mx {

namespace {

constexpr int NB = LU_NB;                   // columns per step (complex K of the update)
constexpr int FT = 128;                     // tile rows (TMEM lanes) = update tile complex columns
constexpr uint32_t F_LBO = 128;             // K-adjacent core matrices
constexpr uint32_t F_SBO = (NB / 4) * 128;  // 8-row groups (1024 B)
constexpr int PLANE = FT * NB * 4;          // one TF32 plane of a 128-row tile: 16 KB
constexpr int TILE = 4 * PLANE;             // re hi, im hi, re lo, im lo: 64 KB
constexpr int IPLANE = NB * NB * 4;         // one TF32 plane of a 32-row operand: 4 KB
constexpr int F_SMEM = 3 * TILE;            // three tile buffers: 192 KB
constexpr int F_WAIT = 1 << 22;             // poll limit of an mbarrier wait
constexpr uint32_t NEG_A = 1u << 13;        // instruction descriptor: negate A
constexpr int THREADS = 512;                // 16 warps: 4 per scheduler to hide latencies
constexpr int MAX_SPAN = 512;               // panel accumulators: 2 x 4 tiles x 64 TMEM columns

__device__ __forceinline__ uint32_t bits_abs(float2 v) { return __float_as_uint(sqrtf(v.x * v.x + v.y * v.y)); }

// one real GEMM: D (+)= A_plane * B_plane^T over K = 32 (four K = 8 instructions)
__device__ __forceinline__ void gemm32(uint32_t d, uint32_t a, uint32_t b, uint32_t id, bool first) {
#pragma unroll
  for (int kk = 0; kk < NB / 8; ++kk)
    tc::mma_tf32(d, tc::sdesc(a + kk * 256, F_LBO, F_SBO), tc::sdesc(b + kk * 256, F_LBO, F_SBO), id,
                 (first && kk == 0) ? 0u : 1u);
}

// complex product of planar operands: Dr (+)= Ar Br - Ai Bi, Di (+)= Ar Bi + Ai Br, each
// factor as hi + lo (planes hi: 0 re, 1 im; lo: 2 re, 3 im); pa / pb: plane strides
template <int SPLIT>
__device__ __forceinline__ void cgemm(uint32_t dr, uint32_t di, uint32_t a, uint32_t pa, uint32_t b, uint32_t pb,
                                      uint32_t idp) {
  const uint32_t idn = idp | NEG_A;
  const uint32_t A0 = a, A1 = a + pa, A2 = a + 2 * pa, A3 = a + 3 * pa;
  const uint32_t B0 = b, B1 = b + pb, B2 = b + 2 * pb, B3 = b + 3 * pb;
  gemm32(dr, A0, B0, idp, true);   // + Ar Br
  gemm32(dr, A1, B1, idn, false);  // - Ai Bi
  gemm32(di, A0, B1, idp, true);   // + Ar Bi
  gemm32(di, A1, B0, idp, false);  // + Ai Br
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
}

// hi / lo planes of four consecutive K values of one operand row
__device__ __forceinline__ void put4(unsigned char* dst, uint32_t plane, uint32_t o, const float2 (&v)[4], bool lo) {
  float hr[4], hi[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    hr[u] = tc::tf32_rn(v[u].x);
    hi[u] = tc::tf32_rn(v[u].y);
  }
  *reinterpret_cast<float4*>(dst + o) = make_float4(hr[0], hr[1], hr[2], hr[3]);
  *reinterpret_cast<float4*>(dst + plane + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
  if (lo) {
    *reinterpret_cast<float4*>(dst + 2 * plane + o) =
        make_float4(v[0].x - hr[0], v[1].x - hr[1], v[2].x - hr[2], v[3].x - hr[3]);
    *reinterpret_cast<float4*>(dst + 3 * plane + o) =
        make_float4(v[0].y - hi[0], v[1].y - hi[1], v[2].y - hi[2], v[3].y - hi[3]);
  }
}

}  // namespace

template <int SPLIT>
__global__ void __launch_bounds__(THREADS, 1) k_band_lu_tc(BandBatch B, float2* A, const int64_t* doff,
                                                          float2* dinv, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ float2 s[NB][NB + 1];   // the diagonal block, then its L and U factors
  __shared__ float2 li[NB][NB + 1];  // L11^{-1}
  __shared__ float2 ui[NB][NB + 1];  // U11^{-1}
  __shared__ __align__(8) uint64_t mbar[3];
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* buf[3] = {smem, smem + TILE, smem + 2 * TILE};
  const uint32_t buf_s[3] = {tc::smem_u32(buf[0]), tc::smem_u32(buf[1]), tc::smem_u32(buf[2])};
  const uint32_t mb[3] = {tc::smem_u32(&mbar[0]), tc::smem_u32(&mbar[1]), tc::smem_u32(&mbar[2])};

  if (tid == 0) {
    for (int q = 0; q < 3; ++q) tc::mbar_init(mb[q], 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;

  uint32_t par[3] = {0u, 0u, 0u};  // parity of the next completion of each barrier
  int my_fail = 0;
  bool failed = false;

  // the CTA factors matrices blockIdx.x, blockIdx.x + gridDim.x, ... (a grid smaller than the
  // batch keeps fewer trailing windows resident at a time)
  for (int m = blockIdx.x; m < B.count && !failed; m += gridDim.x) {
    const int n = B.n[m], b = B.b[m], ld = B.ld[m];
    const int64_t off = B.off[m];
    uint32_t um = 0;  // largest |U| entry this thread finalised (pivot growth)
    __syncthreads();  // the previous matrix's last reads of s, li, ui are done

    for (int k0 = 0; k0 < n && !failed; k0 += NB) {
      const int kb = min(NB, n - k0);
      const int k1 = k0 + kb;
      const int span = min(n - k1, b);
      const int lim = k1 + span;

      // ---- 1. diagonal block: LU, then L11^{-1} and U11^{-1}
      for (int t = tid; t < NB * NB; t += THREADS) {
        const int i = t % NB, j = t / NB;
        float2 v = make_float2(0.f, 0.f);
        if (i < kb && j < kb && abs(i - j) <= b) v = A[bidx(off, ld, b, k0 + i, k0 + j)];
        s[i][j] = v;
        const float2 e = make_float2((i == j && i < kb) ? 1.f : 0.f, 0.f);
        li[i][j] = e;
        ui[i][j] = e;
      }
      __syncthreads();
      for (int k = 0; k < kb; ++k) {
        const float2 piv = s[k][k];
        const float p2 = cabs2(piv);
        if (tid == 0 && !(p2 > 0 && p2 < INFINITY)) atomicAdd(status, 1);
        const float2 inv = crcp(piv);
        __syncthreads();
        for (int i = k + 1 + tid; i < kb; i += THREADS) s[i][k] = cmul(s[i][k], inv);
        __syncthreads();
        // trailing update: warp = column, lane = row (no division by the trailing size)
        const int i = k + 1 + lane;
        if (i < kb)
          for (int j = k + 1 + warp; j < kb; j += THREADS / 32) {
            float2 v = s[i][j];
            cfms(v, s[i][k], s[k][j]);
            s[i][j] = v;
          }
        __syncthreads();
      }
      // L X = I (unit lower, rows top to bottom) and U Y = I (rows bottom to top) by row
      // operations, one row of each per step
      for (int t = 0; t < kb; ++t) {
        const int ku = kb - 1 - t;
        if (tid < NB) ui[ku][tid] = cmul(ui[ku][tid], crcp(s[ku][ku]));
        __syncthreads();
        for (int e = tid; e < 2 * NB * NB; e += THREADS) {
          const int c = e % NB, i = (e / NB) % NB;
          if (e < NB * NB) {
            if (i > t && i < kb) {
              float2 v = li[i][c];
              cfms(v, s[i][t], li[t][c]);
              li[i][c] = v;
            }
          } else if (i < ku) {
            float2 v = ui[i][c];
            cfms(v, s[i][ku], ui[ku][c]);
            ui[i][c] = v;
          }
        }
        __syncthreads();
      }
      // write the factored block and the inverses (column-major [L^{-1}, U^{-1}] blocks, as the
      // local solves read them); stage U11^{-1} and L11^{-1} as the panels' B operands in
      // buf[2]: B[nn][kk] = U11^{-1}(kk, nn) for L21, = L11^{-1}(nn, kk) for U12^T
      float2* dq = dinv + doff[m] + (int64_t)(k0 / NB) * 2 * NB * NB;
      for (int t = tid; t < NB * NB; t += THREADS) {
        const int i = t % NB, j = t / NB;
        if (i < kb && j < kb && abs(i - j) <= b) {
          A[bidx(off, ld, b, k0 + i, k0 + j)] = s[i][j];
          if (i <= j) um = max(um, bits_abs(s[i][j]));
        }
        dq[(int64_t)j * NB + i] = li[i][j];
        dq[NB * NB + (int64_t)j * NB + i] = ui[i][j];
      }
      for (int t = tid; t < 2 * NB * (NB / 4); t += THREADS) {
        const int nn = t % NB, g = (t / NB) % (NB / 4), which = t / (NB * (NB / 4));
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = which == 0 ? ui[4 * g + u][nn] : li[nn][4 * g + u];
        put4(buf[2] + which * 4 * IPLANE, IPLANE, tc::kmaj(nn, 4 * g, F_LBO, F_SBO), v, SPLIT == 3);
      }
      if (span <= 0) break;  // last block column (span is the same for every thread)

      // stage rows [r0, r0 + 128) of A21 / L21 (rows) or columns of A12 / U12 (!rows) into a
      // 128-row operand tile, K = the 32 columns (rows) of the block; a thread's items load first
      constexpr int ITEMS = FT * (NB / 4) / THREADS;
      auto stage = [&](unsigned char* dst, int r0, bool rows) {
        float2 v[ITEMS][4];
#pragma unroll
        for (int it2 = 0; it2 < ITEMS; ++it2) {
          const int t = tid + THREADS * it2;
          const int e = r0 + t % FT, g = t / FT;
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
          const int t = tid + THREADS * it2;
          put4(dst, PLANE, tc::kmaj(t % FT, 4 * (t / FT), F_LBO, F_SBO), v[it2], SPLIT == 3);
        }
      };
      // the same tile staged by warps 1-15 only (warp 0 is issuing products meanwhile)
      constexpr int SW = THREADS - 32;
      constexpr int ITEMS_W = (FT * (NB / 4) + SW - 1) / SW;
      auto stage_w = [&](unsigned char* dst, int r0, bool rows) {
        float2 v[ITEMS_W][4];
#pragma unroll
        for (int it2 = 0; it2 < ITEMS_W; ++it2) {
          const int t = tid - 32 + SW * it2;
          const int e = r0 + t % FT, g = t / FT;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int kc = 4 * g + u, k = k0 + kc;
            v[it2][u] = make_float2(0.f, 0.f);
            if (t < FT * (NB / 4) && kc < kb && e < lim && e - k <= b)
              v[it2][u] = rows ? A[bidx(off, ld, b, e, k)] : A[bidx(off, ld, b, k, e)];
          }
        }
#pragma unroll
        for (int it2 = 0; it2 < ITEMS_W; ++it2) {
          const int t = tid - 32 + SW * it2;
          if (t < FT * (NB / 4)) put4(dst, PLANE, tc::kmaj(t % FT, 4 * (t / FT), F_LBO, F_SBO), v[it2], SPLIT == 3);
        }
      };
      auto wait_bar = [&](int q) -> bool {
        const bool ok = tc::mbar_wait(mb[q], par[q], F_WAIT);
        par[q] ^= 1u;
        tc::fence_after();
        return ok;
      };

      // ---- 2. panels on the tensor cores: tiles p < nt are rows of L21, nt <= p < 2 nt
      // columns of U12, accumulators at TMEM columns 64 p. A two-buffer pipeline: while thread 0
      // issues the products of tile p (buf[p & 1]), warps 1-15 stage tile p + 1 into the other
      // buffer once the products of tile p - 1, which read it, are done (mbarrier p & 1, waited
      // by every thread once per tile, so the per-thread parities stay in step)
      const int nt = (span + FT - 1) / FT;
      const int np = 2 * nt;
      auto panel_row = [&](int p) { return k1 + FT * (p < nt ? p : p - nt); };
      stage(buf[0], panel_row(0), true);
      for (int p = 0; p < np; ++p) {
        tc::fence_proxy_async();
        tc::fence_before();
        if (__syncthreads_or(my_fail)) {
          failed = true;
          break;
        }
        tc::fence_after();
        if (tid == 0) {
          const uint32_t d = tmem + (uint32_t)(64 * p);
          cgemm<SPLIT>(d, d + 32, buf_s[p & 1], PLANE, buf_s[2] + (p < nt ? 0 : 4 * IPLANE), IPLANE,
                       tc::idesc_tf32(FT, NB));
          tc::mma_commit(mb[p & 1]);
        }
        if (p >= 1 && !wait_bar((p - 1) & 1)) my_fail = 1;  // tile p - 1 done: its buffer is free
        if (warp > 0 && p + 1 < np && !my_fail) stage_w(buf[(p + 1) & 1], panel_row(p + 1), p + 1 < nt);
      }
      if (failed) break;
      if (!wait_bar((np - 1) & 1)) my_fail = 1;  // the last tile's products
      // epilogue of the panels: warp w takes TMEM lanes 32 (w % 4) of the tiles p = w / 4 (mod 4)
      {
        const int lg = warp & 3;
        for (int p = warp >> 2; p < np && !my_fail; p += 4) {
          const uint32_t addr = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(64 * p);
          uint32_t vr[32], vi[32];
          tc::tmem_ld32(addr, vr);
          tc::tmem_ld32(addr + 32, vi);
          const int e = k1 + FT * (p < nt ? p : p - nt) + 32 * lg + lane;
          if (e < lim) {
#pragma unroll
            for (int q = 0; q < NB; ++q) {
              const int k = k0 + q;
              if (q < kb && e - k <= b) {
                const float2 x = make_float2(__uint_as_float(vr[q]), __uint_as_float(vi[q]));
                if (p < nt) {
                  A[bidx(off, ld, b, e, k)] = x;
                } else {
                  A[bidx(off, ld, b, k, e)] = x;
                  um = max(um, bits_abs(x));
                }
              }
            }
          }
        }
      }
      tc::fence_before();
      if (__syncthreads_or(my_fail)) {  // L21 and U12 are in place before the update reads them
        failed = true;
        break;
      }
      tc::fence_after();

      // ---- 3. A22 -= L21 U12 over the window, tiles of 128 x 128 complex entries
      // TMEM -> registers -> A22 -= D for tile q (slot q & 1: Re D in columns [0, 128), Im D in
      // [128, 256) of the slot); false if the tensor cores did not finish in time
      auto epilogue = [&](int q) -> bool {
        const int sl = q & 1;
        const int i0 = k1 + FT * (q / nt), j0 = k1 + FT * (q % nt);
        // warp w: TMEM lanes 32 (w % 4) .. (its rows), complex columns 32 (w / 4) .. of the tile
        const int lg = warp & 3, cq = warp >> 2;
        const int i = i0 + 32 * lg + lane;
        const uint32_t base = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(256 * sl) + (uint32_t)(32 * cq);
        const int jb = j0 + 32 * cq;
        // 32 entries of the row in two rounds of 16 (loads of a round first, then its stores);
        // entry (i, jb + u) of the band storage is u (ld - 1) elements after entry (i, jb)
        const bool row_ok = i < lim;
        const int64_t st = ld - 1;
        float2* rp = A + bidx(off, ld, b, row_ok ? i : lim - 1, jb);
        const int nv = row_ok ? min(32, lim - jb) : 0;  // entries of the row inside the window
        // the first round's loads are in flight while the tile's products finish
        float2 x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = u < nv ? rp[u * st] : make_float2(0.f, 0.f);
        if (!wait_bar(sl)) return false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1) {
#pragma unroll
            for (int u = 0; u < 16; ++u) x[u] = 16 + u < nv ? rp[(16 + u) * st] : make_float2(0.f, 0.f);
          }
          uint32_t vr[16], vi[16];
          tc::tmem_ld16(base + 16 * h, vr);
          tc::tmem_ld16(base + 128 + 16 * h, vi);
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (16 * h + u < nv)
              rp[(16 * h + u) * st] = make_float2(x[u].x - __uint_as_float(vr[u]), x[u].y - __uint_as_float(vi[u]));
        }
        return true;
      };

      int pending = -1;
      for (int q = 0; q < nt * nt; ++q) {
        const int it = q / nt, jt = q % nt, sl = q & 1;
        if (jt == 0) {
          if (pending >= 0) {  // the A tile is about to change: its last product must be done
            if (!epilogue(pending)) my_fail = 1;
            pending = -1;
          }
          stage(buf[0], k1 + FT * it, true);
        }
        stage(buf[1 + sl], k1 + FT * jt, false);
        tc::fence_proxy_async();
        tc::fence_before();
        if (__syncthreads_or(my_fail)) {
          failed = true;
          break;
        }
        tc::fence_after();
        if (tid == 0) {
          const uint32_t dr = tmem + (uint32_t)(256 * sl);
          cgemm<SPLIT>(dr, dr + 128, buf_s[0], PLANE, buf_s[1 + sl], PLANE, tc::idesc_tf32(FT, FT));
          tc::mma_commit(mb[sl]);
        }
        if (pending >= 0 && !epilogue(pending)) my_fail = 1;
        pending = q;
      }
      if (!failed && pending >= 0 && !epilogue(pending)) my_fail = 1;
      tc::fence_before();
      if (__syncthreads_or(my_fail)) failed = true;  // the window is updated before the next step
      tc::fence_after();
    }
    if (B.umax) {
      um = __reduce_max_sync(0xffffffffu, um);
      if (lane == 0) atomicMax(B.umax + m, um);
    }
  }

  if (failed && tid == 0) atomicAdd(status + 2, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

bool band_lu_fused_fits(int max_span) { return max_span <= MAX_SPAN; }

void band_lu_fused(const BandBatch& B, float2* A, const int64_t* doff, float2* dinv, int split, int grid,
                   int32_t* status, cudaStream_t s, double bytes, double flops) {
  const int nblk = grid > 0 ? std::min(grid, B.count) : B.count;
  static std::atomic<bool> attr1{false}, attr3{false};
  ProfScope ps(K_LU_UPDATE, s, 1, bytes, flops);
  if (split == 3) {
    if (!attr3) {
      MX_CUDA(cudaFuncSetAttribute(k_band_lu_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM));
      attr3 = true;
    }
    MX_LAUNCH(k_band_lu_tc<3><<<nblk, THREADS, F_SMEM, s>>>(B, A, doff, dinv, status));
  } else {
    if (!attr1) {
      MX_CUDA(cudaFuncSetAttribute(k_band_lu_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM));
      attr1 = true;
    }
    MX_LAUNCH(k_band_lu_tc<1><<<nblk, THREADS, F_SMEM, s>>>(B, A, doff, dinv, status));
  }
  MX_CHECK_LAUNCH();
}

}  // namespace mx

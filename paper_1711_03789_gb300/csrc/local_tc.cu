// Local solves of the additive Schwarz preconditioner (Eq. 3.4) on the tensor cores,
// for the mixed-precision form (c64 factors).
//
// The forward sweep L y = R^l v and the backward sweep U z = y run block column by block
// column (NB = 32). Each step applies the inverted diagonal block to the finished rows of
// the block on the CUDA cores, then updates the rows below (forward) or above (backward)
// within the band as one GEMM: acc(i, :) += F(i, c0:c0+32) x_blk. On the tensor cores
// that GEMM is D += A B^T with
//   A (M = 128): the right-hand-side block in real form; row 2g holds (Re x, -Im x) and
//     row 2g + 1 holds (Im x, Re x) of right-hand side g, interleaved along K = 2 k + c;
//     the TF32 truncation x_hi of x sits in rows [0, 2G), the remainder x - x_hi in rows
//     [LO, LO + 2G), so the products carry x to about FP32 accuracy;
//   B (N = panel rows): the factor panel, row i holding (Re F, Im F)(i, k) along K, stored
//     once at factorisation time as a TF32-rounded image in the K-major core-matrix layout
//     of shared memory and moved by bulk copies;
//   D: tensor memory, lane = real component of a right-hand side, column = row of the
//     matrix modulo 512 (a ring over the rows alive in the band window).
// A row leaves the ring when its block is solved: the block's 32 columns are read back
// (hi + lo lanes), subtracted from the right-hand side and zeroed for reuse.
//
// Warp roles: warps 0-7 run the substitution steps (the elected thread 0 issues the
// MMAs); warp 8 streams the panel chunks (up to 128 rows, 32 KB) through a ring of
// NBUF shared-memory buffers with mbarrier hand-off. Every wait is bounded; a timeout
// sets status[2], stops the block at the next step and drains the copies in flight.
#include "problem.cuh"
#include "tc.cuh"

namespace mx {

namespace {

constexpr int SB = LU_NB;                      // block columns per step (32)
constexpr int KR = 2 * SB;                     // real K per step (64)
constexpr uint32_t LBO = 128;                  // K-adjacent core matrices
constexpr uint32_t SBO = (KR / 4) * 128;       // 8-row groups: 2048 bytes
constexpr int ROW_BYTES = KR * 4;              // one panel row: 256 bytes
constexpr int CHUNK_ROWS = 128;
constexpr int CHUNK_BYTES = CHUNK_ROWS * ROW_BYTES;  // 32 KB
constexpr int NBUF = 5;
constexpr int RING = 512;                      // TMEM columns (accumulator ring)
constexpr int A_BYTES = 128 * ROW_BYTES;       // A operand: 32 KB
constexpr int D_BYTES = SB * SB * 8;           // one inverted diagonal block (c64)
constexpr int MAX_BP = 448;                    // rows alive (<= bp + 2 NB) must fit the ring
constexpr int WAIT_LIMIT = 1 << 22;
constexpr int THREADS = 288;                   // 8 compute warps + 1 copy warp

__host__ __device__ inline int pad32(int x) { return (x + 31) & ~31; }
__host__ __device__ inline int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// Rows [rb, rb + cnt) of the update panel of block s: below the block (dir 0, L) or above
// it (dir 1, U); bp = half-bandwidth rounded up to 32. cnt is a multiple of 32 and may
// include zero rows past the matrix end.
__host__ __device__ inline void panel_rows(int dir, int s, int n, int bp, int& rb, int& cnt) {
  const int c0 = SB * s;
  if (dir == 0) {
    const int c1 = imin(n, c0 + SB);
    rb = c1;
    cnt = pad32(imin(n, c1 + bp) - c1);
  } else {
    rb = imax(0, c0 - bp);
    cnt = c0 - rb;
  }
}

size_t solve_smem_bytes(int G) {
  const int lo = 2 * G > 32 ? 2 * G : 32;
  const int nld = (lo + 2 * G + 31) / 32;
  return (size_t)NBUF * CHUNK_BYTES + A_BYTES + D_BYTES + (size_t)nld * 32 * 32 * 4;
}

}  // namespace

// ---- panel images ---------------------------------------------------------------------
struct PanelArgs {
  BandBatch B;
  const float2* A;         // band LU factors (c64)
  const int64_t* pstart;   // [n_sub + 1] first panel of each subdomain
  const int64_t* ptab;     // byte offset of each panel image
  unsigned char* img;
};

// One block per (subdomain, panel): panel p < nblk is the forward panel of block p,
// p >= nblk the backward panel of block p - nblk. Rows vary fastest so that the band
// columns are read contiguously.
__global__ void k_build_panels(PanelArgs a) {
  const int l = blockIdx.x, p = blockIdx.y;
  const int n = a.B.n[l], b = a.B.b[l], ld = a.B.ld[l];
  const int64_t off = a.B.off[l];
  const int nblk = (n + SB - 1) / SB;
  if (p >= 2 * nblk) return;
  const int dir = p < nblk ? 0 : 1, s = dir ? p - nblk : p;
  int rb, cnt;
  panel_rows(dir, s, n, pad32(b), rb, cnt);
  const int c0 = SB * s, c1 = imin(n, c0 + SB);
  unsigned char* base = a.img + a.ptab[a.pstart[l] + p];
  for (int t = threadIdx.x; t < cnt * SB; t += blockDim.x) {
    const int r = t % cnt, kc = t / cnt;
    const int i = rb + r, k = c0 + kc;
    const bool in = i < n && k < c1 && (dir == 0 ? i - k <= b : k - i <= b);
    const float2 v = in ? a.A[bidx(off, ld, b, i, k)] : make_float2(0.f, 0.f);
    const int o = (r >> 3) * (int)SBO + (kc >> 1) * (int)LBO + (r & 7) * 16 + (kc & 1) * 8;
    *reinterpret_cast<float2*>(base + o) = make_float2(tc::tf32_rn(v.x), tc::tf32_rn(v.y));
  }
}

// Plans and writes the panel images of every subdomain (after the band LU). Subdomains
// whose half-bandwidth exceeds MAX_BP leave the images unbuilt (the CUDA-core solve runs).
void build_panels(Problem& P) {
  P.panels_ok = false;
  if (P.precision != MX_MIXED || !P.factored) return;
  std::vector<int64_t> pstart(P.n_sub + 1, 0), ptab;
  int64_t bytes = 0;
  int maxp = 0;
  for (int l = 0; l < P.n_sub; ++l) {
    const int n = P.h_nl[l], bp = pad32(P.h_band[l]);
    if (bp > MAX_BP) return;
    const int nblk = (n + SB - 1) / SB;
    maxp = std::max(maxp, 2 * nblk);
    pstart[l + 1] = pstart[l] + 2 * nblk;
    for (int p = 0; p < 2 * nblk; ++p) {
      const int dir = p < nblk ? 0 : 1, s = dir ? p - nblk : p;
      int rb, cnt;
      panel_rows(dir, s, n, bp, rb, cnt);
      ptab.push_back(bytes);
      bytes += (int64_t)cnt * ROW_BYTES;
    }
  }
  cudaStream_t s = P.stream;
  P.pan_start.alloc(P.n_sub + 1);
  P.pan_tab.alloc(std::max<size_t>(1, ptab.size()));
  P.panels.alloc(std::max<int64_t>(bytes, 16));
  MX_CUDA(cudaMemcpyAsync(P.pan_start.p, pstart.data(), pstart.size() * 8, cudaMemcpyHostToDevice, s));
  if (!ptab.empty())
    MX_CUDA(cudaMemcpyAsync(P.pan_tab.p, ptab.data(), ptab.size() * 8, cudaMemcpyHostToDevice, s));
  PanelArgs a{BandBatch{P.n_sub, P.nl.p, P.band.p, P.ld.p, P.mat_off.p}, reinterpret_cast<const float2*>(P.factors.p),
              P.pan_start.p, P.pan_tab.p, P.panels.p};
  if (maxp > 0) {
    ProfScope ps(K_LAYOUT, s);
    MX_LAUNCH(k_build_panels<<<dim3(P.n_sub, maxp), 256, 0, s>>>(a));
    MX_CHECK_LAUNCH();
  }
  MX_CUDA(cudaStreamSynchronize(s));
  P.panel_bytes = bytes;
  P.panels_ok = true;
}

// Device bytes build_panels will allocate (0 if the images cannot be used).
int64_t panel_bytes_planned(const Problem& P) {
  if (P.precision != MX_MIXED) return 0;
  int64_t bytes = 0;
  for (int l = 0; l < P.n_sub; ++l) {
    const int n = P.h_nl[l], bp = pad32(P.h_band[l]);
    if (bp > MAX_BP) return 0;
    const int nblk = (n + SB - 1) / SB;
    for (int p = 0; p < 2 * nblk; ++p) {
      const int dir = p < nblk ? 0 : 1, s = dir ? p - nblk : p;
      int rb, cnt;
      panel_rows(dir, s, n, bp, rb, cnt);
      bytes += (int64_t)cnt * ROW_BYTES;
    }
  }
  return bytes;
}

// ---- the solve kernel ----------------------------------------------------------------------
struct TcArgs {
  int nrhs;
  const int64_t* offsets;
  const int32_t* lists;
  const int32_t* nl;
  const int32_t* band;
  const unsigned char* img;
  const int64_t* pstart;
  const int64_t* ptab;
  const float2* dinv;
  const int64_t* doff;
  const void* v;  // [n][nrhs] c128 (vtype 0) or c64 (vtype 1)
  int vtype;
  float2* out;    // [sum_local][nrhs]
  int32_t* status;
};

__device__ __forceinline__ float2 load_rhs(const void* v, int vtype, int64_t idx) {
  if (vtype == 0) {
    const double2 d = reinterpret_cast<const double2*>(v)[idx];
    return make_float2((float)d.x, (float)d.y);
  }
  return reinterpret_cast<const float2*>(v)[idx];
}

template <int G>
__global__ void __launch_bounds__(THREADS, 1) k_local_solve_tc(TcArgs a) {
  constexpr int LO = 2 * G > 32 ? 2 * G : 32;     // first lane / A row of the low parts
  constexpr int NLD = (LO + 2 * G + 31) / 32;     // warps reading accumulator lanes
  constexpr int PAIRS = SB * G / 256;             // (row, rhs) pairs per compute thread
  static_assert(SB * G % 256 == 0 && LO + 2 * G <= 128, "unsupported group size");

  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* bufs = smem;
  unsigned char* Aop = smem + NBUF * CHUNK_BYTES;
  float2* Dsm = reinterpret_cast<float2*>(Aop + A_BYTES);
  float* accs = reinterpret_cast<float*>(Aop + A_BYTES + D_BYTES);  // [NLD][32 rows][32 lanes]
  float2* vs = reinterpret_cast<float2*>(accs);                     // [32][G], reuses accs
  __shared__ __align__(8) uint64_t full[NBUF], empty[NBUF], mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int cerr;  // set by compute threads only, read after barrier B

  const int groups = (a.nrhs + G - 1) / G;
  const int l = blockIdx.x / groups, g0 = (blockIdx.x % groups) * G;
  const int gn = imin(G, a.nrhs - g0);
  const int n = a.nl[l], bp = pad32(a.band[l]);
  const int nblk = (n + SB - 1) / SB;
  const int64_t pos0 = a.offsets[l];
  const int64_t pbase = a.pstart[l];
  const float2* Dl = a.dinv + a.doff[l];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bufs_a = tc::smem_u32(bufs), A_a = tc::smem_u32(Aop);
  const uint32_t full_a = tc::smem_u32(&full[0]), empty_a = tc::smem_u32(&empty[0]);
  const uint32_t mma_a = tc::smem_u32(&mma_bar);

  if (tid == 0) {
    for (int i = 0; i < NBUF; ++i) {
      tc::mbar_init(full_a + 8 * i, 1);
      tc::mbar_init(empty_a + 8 * i, 1);
    }
    tc::mbar_init(mma_a, 1);
    tc::mbar_fence_init();
    cerr = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), RING);
  for (int t = tid; t < A_BYTES / 16; t += THREADS) reinterpret_cast<float4*>(Aop)[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  // the ring starts at zero in every lane that is read back
  if (warp < NLD)
    for (int c = 0; c < RING; c += 32) tc::tmem_zero32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();

  if (warp == 8) {
    // ---- copy warp: every panel chunk of both sweeps, in consumption order
    if (lane == 0) {
      int it = 0;
      bool stop = false;
      for (int dir = 0; dir < 2 && !stop; ++dir)
        for (int q = 0; q < nblk && !stop; ++q) {
          const int s = dir == 0 ? q : nblk - 1 - q;
          int rb, cnt;
          panel_rows(dir, s, n, bp, rb, cnt);
          const unsigned char* src = a.img + a.ptab[pbase + (dir ? nblk + s : s)];
          for (int r0 = 0; r0 < cnt; r0 += CHUNK_ROWS) {
            const int nr = imin(CHUNK_ROWS, cnt - r0);
            const int buf = it % NBUF, use = it / NBUF;
            if (cerr) { stop = true; break; }
            if (use > 0 && !tc::mbar_wait(empty_a + 8 * buf, (use - 1) & 1, WAIT_LIMIT)) {
              atomicAdd(a.status + 2, 1);
              stop = true;
              break;
            }
            tc::mbar_expect_tx(full_a + 8 * buf, (uint32_t)(nr * ROW_BYTES));
            tc::bulk_g2s(bufs_a + buf * CHUNK_BYTES, src + (int64_t)r0 * ROW_BYTES, (uint32_t)(nr * ROW_BYTES),
                         full_a + 8 * buf);
            ++it;
          }
        }
      // no copy may still be in flight when the block exits
      for (int j = imax(0, it - NBUF); j < it; ++j) tc::mbar_wait(full_a + 8 * (j % NBUF), (j / NBUF) & 1, WAIT_LIMIT);
    }
  } else {
    // ---- compute warps
    float2 rpre[PAIRS];
    float4 dpre[2];
    auto prefetch = [&](int dir, int s) {
      const int c0 = SB * s;
#pragma unroll
      for (int c = 0; c < PAIRS; ++c) {
        const int t = tid + 256 * c, j = t / G, g = t % G, i = c0 + j;
        float2 r = make_float2(0.f, 0.f);
        if (i < n && g < gn) {
          r = dir == 0 ? load_rhs(a.v, a.vtype, (int64_t)a.lists[pos0 + i] * a.nrhs + g0 + g)
                       : a.out[(pos0 + i) * a.nrhs + g0 + g];
        }
        rpre[c] = r;
      }
      const float4* D4 = reinterpret_cast<const float4*>(Dl + (int64_t)s * 2 * SB * SB + dir * SB * SB);
      dpre[0] = D4[tid];
      dpre[1] = D4[tid + 256];
    };
    if (nblk > 0) prefetch(0, 0);
    bool pending = false, stop = false;
    uint32_t mma_par = 0;
    int it = 0;  // chunk counter (thread 0)
    for (int dir = 0; dir < 2 && !stop; ++dir) {
      for (int q = 0; q < nblk; ++q) {
        const int s = dir == 0 ? q : nblk - 1 - q;
        const int c0 = SB * s, kb = imin(SB, n - c0);
        tc::bar_sync(1, 256);  // A
        if (pending) {
          if (!tc::mbar_wait(mma_a, mma_par, WAIT_LIMIT)) {
            cerr = 1;
            if (tid == 0) atomicAdd(a.status + 2, 1);
          }
          mma_par ^= 1;
          pending = false;
          tc::fence_after();
        }
        // retire the block rows from the ring
        if (warp < NLD) {
          uint32_t r[32];
          const uint32_t ad = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(c0 & (RING - 1));
          tc::tmem_ld32(ad, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) accs[(warp * 32 + j) * 32 + lane] = __uint_as_float(r[j]);
          tc::tmem_zero32(ad);
        }
        reinterpret_cast<float4*>(Dsm)[tid] = dpre[0];
        reinterpret_cast<float4*>(Dsm)[tid + 256] = dpre[1];
        tc::bar_sync(1, 256);  // B
        if (cerr) { stop = true; break; }
        // v = r - (acc_hi + acc_lo)
        float2 vv[PAIRS];
#pragma unroll
        for (int c = 0; c < PAIRS; ++c) {
          const int t = tid + 256 * c, j = t / G, g = t % G;
          auto acc = [&](int L) { return accs[((L >> 5) * 32 + j) * 32 + (L & 31)]; };
          const float re = acc(2 * g) + acc(LO + 2 * g), im = acc(2 * g + 1) + acc(LO + 2 * g + 1);
          vv[c] = make_float2(rpre[c].x - re, rpre[c].y - im);
        }
        tc::bar_sync(1, 256);
#pragma unroll
        for (int c = 0; c < PAIRS; ++c) {
          const int t = tid + 256 * c;
          vs[(t / G) * G + t % G] = vv[c];
        }
        tc::bar_sync(1, 256);
        // x_blk = D v (D zero outside the kb x kb block), written out and staged as A
#pragma unroll
        for (int c = 0; c < PAIRS; ++c) {
          const int t = tid + 256 * c, i = t / G, g = t % G;
          CAcc2 sacc;
          cacc_zero(sacc);
#pragma unroll 8
          for (int jj = 0; jj < SB; ++jj) cacc(sacc, Dsm[i + SB * jj], vs[jj * G + g]);
          const float2 x = cacc_value(sacc);
          if (i < kb && g < gn) a.out[(pos0 + c0 + i) * a.nrhs + g0 + g] = x;
          const float2 h = make_float2(tc::tf32_hi(x.x), tc::tf32_hi(x.y));
          const float2 e = make_float2(x.x - h.x, x.y - h.y);
          *reinterpret_cast<float2*>(Aop + tc::kmaj(2 * g, 2 * i, LBO, SBO)) = make_float2(h.x, -h.y);
          *reinterpret_cast<float2*>(Aop + tc::kmaj(2 * g + 1, 2 * i, LBO, SBO)) = make_float2(h.y, h.x);
          *reinterpret_cast<float2*>(Aop + tc::kmaj(LO + 2 * g, 2 * i, LBO, SBO)) = make_float2(e.x, -e.y);
          *reinterpret_cast<float2*>(Aop + tc::kmaj(LO + 2 * g + 1, 2 * i, LBO, SBO)) = make_float2(e.y, e.x);
        }
        tc::fence_proxy_async();
        tc::fence_before();
        tc::bar_sync(1, 256);  // D
        // next block's right-hand side and diagonal block (y of this block is visible now)
        if (dir == 0) {
          if (q + 1 < nblk) prefetch(0, s + 1);
          else prefetch(1, nblk - 1);
        } else if (q + 1 < nblk) {
          prefetch(1, s - 1);
        }
        int rb, cnt;
        panel_rows(dir, s, n, bp, rb, cnt);
        if (cnt > 0) {
          if (tid == 0) {
            tc::fence_after();
            for (int r0 = 0; r0 < cnt; r0 += CHUNK_ROWS) {
              const int nr = imin(CHUNK_ROWS, cnt - r0);
              const int buf = it % NBUF, use = it / NBUF;
              if (tc::mbar_wait(full_a + 8 * buf, use & 1, WAIT_LIMIT)) {
                const uint32_t b0 = bufs_a + buf * CHUNK_BYTES;
                int done = 0;
                while (done < nr) {
                  const int col = (rb + r0 + done) & (RING - 1);
                  const int nn = imin(nr - done, RING - col);
                  const uint32_t idesc = tc::idesc_tf32(128, nn);
#pragma unroll
                  for (int kk = 0; kk < KR / 8; ++kk)
                    tc::mma_tf32(tmem + (uint32_t)col, tc::sdesc(A_a + kk * 256, LBO, SBO),
                                 tc::sdesc(b0 + (done >> 3) * SBO + kk * 256, LBO, SBO), idesc, 1);
                  done += nn;
                }
              } else {
                cerr = 1;
                atomicAdd(a.status + 2, 1);
              }
              tc::mma_commit(empty_a + 8 * buf);
              ++it;
            }
            tc::mma_commit(mma_a);
          }
          pending = true;
        }
      }
    }
    if (pending && !tc::mbar_wait(mma_a, mma_par, WAIT_LIMIT) && tid == 0) atomicAdd(a.status + 2, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, RING);
  }
}

template <int G>
static void launch_tc(const TcArgs& a, int n_sub, cudaStream_t s, double alg_bytes, double alg_flops) {
  const size_t smem = solve_smem_bytes(G);
  static bool configured = false;
  if (!configured) {
    MX_CUDA(cudaFuncSetAttribute(k_local_solve_tc<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  const int groups = (a.nrhs + G - 1) / G;
  ProfScope ps(K_LOCAL_SOLVE, s, 1, alg_bytes, alg_flops);
  MX_LAUNCH(k_local_solve_tc<G><<<n_sub * groups, THREADS, smem, s>>>(a));
  MX_CHECK_LAUNCH();
}

// z_l = (A^l)^{-1} R^l v on the tensor cores (mixed form; panels built)
void local_solves_tc(Problem& P, const void* v, int vtype, void* loc, int nrhs, double alg_bytes, double alg_flops) {
  MX_REQUIRE(P.panels_ok, MX_EINVAL, "tensor-core local solve without panel images");
  TcArgs a{};
  a.nrhs = nrhs;
  a.offsets = P.offsets.p;
  a.lists = P.lists.p;
  a.nl = P.nl.p;
  a.band = P.band.p;
  a.img = P.panels.p;
  a.pstart = P.pan_start.p;
  a.ptab = P.pan_tab.p;
  a.dinv = reinterpret_cast<const float2*>(P.dinv.p);
  a.doff = P.dinv_off.p;
  a.v = v;
  a.vtype = vtype;
  a.out = reinterpret_cast<float2*>(loc);
  a.status = P.status.p;
  if (nrhs <= 8) launch_tc<8>(a, P.n_sub, P.stream, alg_bytes, alg_flops);
  else if (nrhs <= 16) launch_tc<16>(a, P.n_sub, P.stream, alg_bytes, alg_flops);
  else launch_tc<32>(a, P.n_sub, P.stream, alg_bytes, alg_flops);
}

}  // namespace mx

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
// Warp roles: warps 0-7 run the substitution steps; warp 9 issues the MMAs of a step as
// soon as its A operand is staged (the 32 rows the next block needs first, so the rest of
// the update runs on the tensor cores while the next block is solved); warp 8 streams the
// panel chunks (up to 128 rows, 32 KB) through a ring of shared-memory buffers and the
// inverted diagonal blocks through a second ring, with mbarrier hand-off. Every wait is
// bounded; a timeout sets status[2], stops the block at the next step and drains the
// copies in flight.
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
constexpr int RING = 512;                      // TMEM columns (accumulator ring)
constexpr int A_BYTES = 128 * ROW_BYTES;       // A operand: 32 KB
constexpr int D_BYTES = SB * SB * 8;           // one inverted diagonal block (c64)
constexpr int MAX_BP = 448;                    // rows alive (<= bp + 2 NB) must fit the ring
constexpr int WAIT_LIMIT = 1 << 22;
constexpr int THREADS = 320;                   // 8 compute warps, 1 copy warp, 1 MMA warp

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
  const void* v;  // [n][nrhs] c128 (vtype 0), c64 (1) or complex double-float (3)
  int vtype;
  float2* out;    // [sum_local][nrhs]
  int32_t* status;
};

__device__ __forceinline__ float2 load_rhs(const void* v, int vtype, int64_t idx) {
  if (vtype == 0) {
    const double2 d = reinterpret_cast<const double2*>(v)[idx];
    return make_float2((float)d.x, (float)d.y);
  }
  if (vtype == 3) {  // complex double-float: the c64 rounding is the high half
    const float4 d = reinterpret_cast<const float4*>(v)[idx];
    return make_float2(d.x, d.y);
  }
  return reinterpret_cast<const float2*>(v)[idx];
}

template <int G>
struct TcCfg {
  static constexpr int LO = 2 * G > 32 ? 2 * G : 32;       // first lane / A row of the low parts
  static constexpr int NLD = (LO + 2 * G + 31) / 32;       // warps reading accumulator lanes
  static constexpr int UNITS = 16 * G;                     // (row pair, rhs) units per block step
  static constexpr int UPT = UNITS >= 256 ? UNITS / 256 : 1;
  static constexpr int NBUF = G >= 32 ? 3 : 4;             // panel chunk buffers
  static constexpr size_t OFF_A = (size_t)NBUF * CHUNK_BYTES;
  static constexpr size_t OFF_D = OFF_A + 2 * A_BYTES;
  static constexpr size_t OFF_ACC = OFF_D + 2 * D_BYTES;
  static constexpr size_t OFF_VS = OFF_ACC + (size_t)NLD * 32 * 32 * 4;
  static constexpr size_t SMEM = OFF_VS + (size_t)SB * G * 8;
};

// A operand row (TMEM lane) of real component ri of right-hand side g, part 0 = TF32 hi,
// part 1 = remainder: eight consecutive right-hand sides share a core matrix, so the
// 16-byte stores of eight threads hit eight different bank groups.
template <int G>
__device__ __forceinline__ int arow(int g, int ri, int part) {
  return part * TcCfg<G>::LO + 16 * (g >> 3) + 8 * ri + (g & 7);
}

// MMAs for `len` panel rows starting at row `off` of the chunk in shared memory at b0,
// matrix row `row0` first; split where the accumulator ring wraps.
__device__ __forceinline__ void mma_rows(uint32_t tmem, uint64_t da, uint32_t b0, int off, int len, int row0) {
  while (len > 0) {
    const int col = row0 & (RING - 1);
    const int nn = imin(len, RING - col);
    const uint32_t idesc = tc::idesc_tf32(128, nn);
    const uint64_t db = tc::sdesc(b0 + (uint32_t)(off >> 3) * SBO, LBO, SBO);
#pragma unroll
    for (int kk = 0; kk < KR / 8; ++kk) tc::mma_tf32(tmem + (uint32_t)col, da + 16 * kk, db + 16 * kk, idesc, 1);
    off += nn;
    row0 += nn;
    len -= nn;
  }
}

template <int G>
__global__ void __launch_bounds__(THREADS, 1) k_local_solve_tc(TcArgs a) {
  using C = TcCfg<G>;
  constexpr int LO = C::LO, NLD = C::NLD, UNITS = C::UNITS, UPT = C::UPT, NBUF = C::NBUF;
  static_assert(G % 8 == 0 && LO + 2 * G <= 128, "unsupported group size");

  extern __shared__ __align__(1024) unsigned char smem[];
  float* accs = reinterpret_cast<float*>(smem + C::OFF_ACC);  // [32 rows][NLD * 32 lanes]
  float2* vs = reinterpret_cast<float2*>(smem + C::OFF_VS);   // [32 rows][G]
  __shared__ __align__(8) uint64_t full[NBUF], empty[NBUF], dfull[2], dempty[2], mma_bar, aready;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int cerr;   // set by compute threads only, read after barrier B
  __shared__ volatile int merr;   // set by the MMA warp, folded into cerr by thread 0

  const int groups = (a.nrhs + G - 1) / G;
  const int l = blockIdx.x / groups, g0 = (blockIdx.x % groups) * G;
  const int gn = imin(G, a.nrhs - g0);
  const int n = a.nl[l], bp = pad32(a.band[l]);
  const int nblk = (n + SB - 1) / SB;
  const int64_t pos0 = a.offsets[l];
  const int64_t pbase = a.pstart[l];
  const float2* Dl = a.dinv + a.doff[l];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bufs_a = tc::smem_u32(smem), A_a = bufs_a + (uint32_t)C::OFF_A;
  const uint32_t D_a = bufs_a + (uint32_t)C::OFF_D;
  const uint32_t full_a = tc::smem_u32(&full[0]), empty_a = tc::smem_u32(&empty[0]);
  const uint32_t dfull_a = tc::smem_u32(&dfull[0]), dempty_a = tc::smem_u32(&dempty[0]);
  const uint32_t mma_a = tc::smem_u32(&mma_bar), aready_a = tc::smem_u32(&aready);

  if (tid == 0) {
    for (int i = 0; i < NBUF; ++i) {
      tc::mbar_init(full_a + 8 * i, 1);
      tc::mbar_init(empty_a + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(dfull_a + 8 * i, 1);
      tc::mbar_init(dempty_a + 8 * i, 1);
    }
    tc::mbar_init(mma_a, 1);
    tc::mbar_init(aready_a, 1);
    tc::mbar_fence_init();
    cerr = 0;
    merr = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), RING);
  {
    float4* A4 = reinterpret_cast<float4*>(smem + C::OFF_A);
    for (int t = tid; t < 2 * A_BYTES / 16; t += THREADS) A4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
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
    if (lane == 0) {
      // ---- panel chunks of both sweeps in consumption order (backward panels bottom-up)
      int it = 0;
      bool stop = false;
      for (int dir = 0; dir < 2 && !stop; ++dir)
        for (int q = 0; q < nblk && !stop; ++q) {
          const int s = dir == 0 ? q : nblk - 1 - q;
          int rb, cnt;
          panel_rows(dir, s, n, bp, rb, cnt);
          const unsigned char* src = a.img + a.ptab[pbase + (dir ? nblk + s : s)];
          const int nch = (cnt + CHUNK_ROWS - 1) / CHUNK_ROWS;
          for (int k = 0; k < nch; ++k) {
            const int ch = dir == 0 ? k : nch - 1 - k;
            const int r0 = ch * CHUNK_ROWS, nr = imin(CHUNK_ROWS, cnt - r0);
            const int buf = it % NBUF, use = it / NBUF;
            if (cerr || merr) { stop = true; break; }
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
      for (int j = imax(0, it - NBUF); j < it; ++j) tc::mbar_wait(full_a + 8 * (j % NBUF), (j / NBUF) & 1, WAIT_LIMIT);
    } else if (lane == 1) {
      // ---- inverted diagonal blocks, one step ahead
      int ss = 0;
      for (int dir = 0; dir < 2; ++dir)
        for (int q = 0; q < nblk; ++q, ++ss) {
          const int s = dir == 0 ? q : nblk - 1 - q;
          const int st = ss & 1, use = ss >> 1;
          if (cerr || merr) break;
          if (use > 0 && !tc::mbar_wait(dempty_a + 8 * st, (use - 1) & 1, WAIT_LIMIT)) {
            atomicAdd(a.status + 2, 1);
            break;
          }
          tc::mbar_expect_tx(dfull_a + 8 * st, (uint32_t)D_BYTES);
          tc::bulk_g2s(D_a + st * D_BYTES, Dl + (int64_t)s * 2 * SB * SB + dir * SB * SB, (uint32_t)D_BYTES,
                       dfull_a + 8 * st);
        }
      for (int j = imax(0, ss - 2); j < ss; ++j) tc::mbar_wait(dfull_a + 8 * (j & 1), (j >> 1) & 1, WAIT_LIMIT);
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // ---- MMA issue: per step, once the compute warps have staged the A operand, the
      // 32 rows the next block needs first (then the mma_bar commit), then the rest
      int it = 0, ss = 0;
      bool failed = false;
      for (int dir = 0; dir < 2; ++dir) {
        bool stop = false;
        for (int q = 0; q < nblk; ++q, ++ss) {
          const int s = dir == 0 ? q : nblk - 1 - q;
          int rb, cnt;
          panel_rows(dir, s, n, bp, rb, cnt);
          if (!tc::mbar_wait_flag(aready_a, ss & 1, WAIT_LIMIT, &cerr)) { stop = true; break; }
          tc::fence_after();
          if (cnt == 0 || failed) {
            tc::mma_commit(mma_a);
            continue;
          }
          const uint64_t da = tc::sdesc(A_a + (uint32_t)((ss & 1) * A_BYTES), LBO, SBO);
          const int nch = (cnt + CHUNK_ROWS - 1) / CHUNK_ROWS;
          for (int k = 0; k < nch; ++k) {
            const int ch = dir == 0 ? k : nch - 1 - k;
            const int r0 = ch * CHUNK_ROWS, nr = imin(CHUNK_ROWS, cnt - r0);
            const int buf = it % NBUF, use = it / NBUF;
            const uint32_t b0 = bufs_a + buf * CHUNK_BYTES;
            const bool ok = !failed && tc::mbar_wait(full_a + 8 * buf, use & 1, WAIT_LIMIT);
            if (!ok && !failed) {
              failed = true;
              merr = 1;
              atomicAdd(a.status + 2, 1);
            }
            if (k == 0) {
              const int fr = dir == 0 ? 0 : cnt - 32 - r0;
              if (ok) mma_rows(tmem, da, b0, fr, 32, rb + r0 + fr);
              tc::mma_commit(mma_a);
              if (ok && fr > 0) mma_rows(tmem, da, b0, 0, fr, rb + r0);
              if (ok && nr - fr - 32 > 0) mma_rows(tmem, da, b0, fr + 32, nr - fr - 32, rb + r0 + fr + 32);
            } else if (ok) {
              mma_rows(tmem, da, b0, 0, nr, rb + r0);
            }
            if (ok) tc::mma_commit(empty_a + 8 * buf);
            ++it;
          }
        }
        if (stop) break;
      }
    }
  } else {
    // ---- compute warps
    float2 rcur[UPT][2], rnext[UPT][2];
    auto load_r = [&](float2 (&r)[UPT][2], int dir, int s) {
      const int c0 = SB * s;
#pragma unroll
      for (int u = 0; u < UPT; ++u) {
        const int t = tid + 256 * u, p = t / G, g = t % G;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int i = c0 + 2 * p + e;
          float2 v = make_float2(0.f, 0.f);
          if (t < UNITS && i < n && g < gn)
            v = dir == 0 ? load_rhs(a.v, a.vtype, (int64_t)a.lists[pos0 + i] * a.nrhs + g0 + g)
                         : a.out[(pos0 + i) * a.nrhs + g0 + g];
          r[u][e] = v;
        }
      }
    };
    if (nblk > 0) load_r(rcur, 0, 0);
    bool pending = false, stop = false;
    uint32_t mma_par = 0;
    int ss = 0;
    for (int dir = 0; dir < 2 && !stop; ++dir) {
      for (int q = 0; q < nblk; ++q, ++ss) {
        const int s = dir == 0 ? q : nblk - 1 - q;
        const int c0 = SB * s, kb = imin(SB, n - c0);
        const bool transition = dir == 0 && q == nblk - 1;
        // right-hand side of the next block, a full step ahead (at the turn of the sweeps
        // it is this block's y, taken from the registers below)
        if (!transition) {
          if (dir == 0) load_r(rnext, 0, s + 1);
          else if (q + 1 < nblk) load_r(rnext, 1, s - 1);
        }
        // retire the block rows from the ring (the warps that own their lanes)
        if (warp < NLD) {
          if (pending && !tc::mbar_wait(mma_a, mma_par, WAIT_LIMIT)) {
            cerr = 1;
            if (lane == 0) atomicAdd(a.status + 2, 1);
          }
          if (tid == 0 && merr) cerr = 1;
          tc::fence_after();
          uint32_t r[32];
          const uint32_t ad = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(c0 & (RING - 1));
          tc::tmem_ld32(ad, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) accs[j * (32 * NLD) + warp * 32 + lane] = __uint_as_float(r[j]);
          tc::tmem_zero32(ad);
        }
        if (pending) {
          mma_par ^= 1;
          pending = false;
        }
        tc::bar_sync(1, 256);  // B
        if (cerr) { stop = true; break; }
        // v = r - (acc_hi + acc_lo)
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          const int t = tid + 256 * u, p = t / G, g = t % G;
          if (t < UNITS) {
            const int mr = arow<G>(g, 0, 0), mi = arow<G>(g, 1, 0), lr = arow<G>(g, 0, 1), li = arow<G>(g, 1, 1);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int j = 2 * p + e;
              const float* row = accs + j * (32 * NLD);
              vs[j * G + g] = make_float2(rcur[u][e].x - (row[mr] + row[lr]), rcur[u][e].y - (row[mi] + row[li]));
            }
          }
        }
        tc::bar_sync(1, 256);  // C
        // x_blk = D v (D zero outside the kb x kb block), written out and staged as A
        const int st = ss & 1;
        if (!tc::mbar_wait(dfull_a + 8 * st, (ss >> 1) & 1, WAIT_LIMIT)) {
          cerr = 1;
          if (tid == 0) atomicAdd(a.status + 2, 1);
        }
        const float4* D4 = reinterpret_cast<const float4*>(smem + C::OFF_D + st * D_BYTES);
        unsigned char* Ab = smem + C::OFF_A + (ss & 1) * A_BYTES;
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          const int t = tid + 256 * u, p = t / G, g = t % G;
          if (t < UNITS) {
            CAcc2 s0, s1;
            cacc_zero(s0);
            cacc_zero(s1);
#pragma unroll 8
            for (int jj = 0; jj < SB; ++jj) {
              const float4 d = D4[p + (SB / 2) * jj];  // D(2p, jj), D(2p + 1, jj)
              const float2 w = vs[jj * G + g];
              cacc(s0, make_float2(d.x, d.y), w);
              cacc(s1, make_float2(d.z, d.w), w);
            }
            const float2 x0 = cacc_value(s0), x1 = cacc_value(s1);
            if (g < gn) {
              if (2 * p < kb) a.out[(pos0 + c0 + 2 * p) * a.nrhs + g0 + g] = x0;
              if (2 * p + 1 < kb) a.out[(pos0 + c0 + 2 * p + 1) * a.nrhs + g0 + g] = x1;
            }
            if (transition) {
              rnext[u][0] = x0;
              rnext[u][1] = x1;
            }
            const float2 h0 = make_float2(tc::tf32_hi(x0.x), tc::tf32_hi(x0.y));
            const float2 h1 = make_float2(tc::tf32_hi(x1.x), tc::tf32_hi(x1.y));
            const float2 e0 = make_float2(x0.x - h0.x, x0.y - h0.y);
            const float2 e1 = make_float2(x1.x - h1.x, x1.y - h1.y);
            const int k4 = 4 * p;
            *reinterpret_cast<float4*>(Ab + tc::kmaj(arow<G>(g, 0, 0), k4, LBO, SBO)) = make_float4(h0.x, -h0.y, h1.x, -h1.y);
            *reinterpret_cast<float4*>(Ab + tc::kmaj(arow<G>(g, 1, 0), k4, LBO, SBO)) = make_float4(h0.y, h0.x, h1.y, h1.x);
            *reinterpret_cast<float4*>(Ab + tc::kmaj(arow<G>(g, 0, 1), k4, LBO, SBO)) = make_float4(e0.x, -e0.y, e1.x, -e1.y);
            *reinterpret_cast<float4*>(Ab + tc::kmaj(arow<G>(g, 1, 1), k4, LBO, SBO)) = make_float4(e0.y, e0.x, e1.y, e1.x);
          }
        }
        tc::fence_proxy_async();
        tc::fence_before();
        tc::bar_sync(1, 256);  // D
        if (tid == 0) {
          tc::mbar_arrive(dempty_a + 8 * st);  // diagonal block consumed
          tc::mbar_arrive(aready_a);            // A operand of this step staged
        }
        pending = true;
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          rcur[u][0] = rnext[u][0];
          rcur[u][1] = rnext[u][1];
        }
      }
    }
    // the last step's commit covers every MMA: all have completed before the tensor
    // memory is released
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
  const size_t smem = TcCfg<G>::SMEM;
  static std::atomic<bool> configured{false};
  if (!configured) {
    MX_CUDA(cudaFuncSetAttribute(k_local_solve_tc<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  const int groups = (a.nrhs + G - 1) / G;
  ProfScope ps(K_LOCAL_SOLVE, s, 1, alg_bytes, alg_flops);
  MX_LAUNCH(k_local_solve_tc<G><<<n_sub * groups, THREADS, smem, s>>>(a));
  MX_CHECK_LAUNCH();
}

// Failure-path probe. Thread 0 of every block initialises an mbarrier that nothing ever
// arrives on and waits on it with the bounded wait of the tensor-core kernels (`limit`
// polls); the wait runs out and the block adds one to status[2], as a timed-out wait in a
// real kernel does, then returns. The block holds no tensor memory and has no copies in
// flight, so nothing is left to drain.
__global__ void k_wait_probe(int limit, int32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = tc::smem_u32(&bar);
  if (threadIdx.x == 0) {
    tc::mbar_init(a, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(a, 0, limit)) atomicAdd(status + 2, 1);
}

int32_t wait_probe(Problem& P, int limit, int blocks) {
  cudaStream_t s = P.stream;
  MX_CUDA(cudaMemsetAsync(P.status.p + 2, 0, sizeof(int32_t), s));
  MX_LAUNCH(k_wait_probe<<<blocks, 32, 0, s>>>(limit, P.status.p));
  MX_CHECK_LAUNCH();
  int32_t timeouts = 0;
  MX_CUDA(cudaMemcpyAsync(&timeouts, P.status.p + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  return timeouts;
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

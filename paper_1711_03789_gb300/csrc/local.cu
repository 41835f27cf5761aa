// Local subdomain matrices A^l = R^l A_{xi_prec} (R^l)^T (Eq. 3.3), their batched LU
// factorisation and the local solves of the additive Schwarz preconditioner (Eq. 3.4).
//
// Storage. In the vertex-major DOF order each minor is banded with half-bandwidth b_l
// (a few hundred for 5^3-cell boxes, against n_l ~ 2000). LU without pivoting creates no
// fill outside the band of a banded matrix, so the band-limited factorisation below
// produces exactly the factors of the dense no-pivot LU; the entries it skips are exact
// zeros. Matrices are stored LAPACK-band style: element (i, j), |i - j| <= b, at
//   off_l + j * ldab_l + (b_l + i - j),   ldab_l = 2 b_l + 1 rounded up to a multiple of 4,
// so every column's band is contiguous. Coercivity (Lemma 2.2) keeps every pivot of the
// no-pivot LU away from zero for xi_prec != 0 (Sec. 3.3).
//
// Factorisation: right-looking blocked LU over the band, NB columns per step, three
// kernels per step for the whole batch (diagonal block, panels, trailing update).
// Local solves: forward/backward substitution on the band with a sliding window of the
// right-hand side block in shared memory; the gather R^l v is fused into the window load.
#include <type_traits>

#include "problem.cuh"

namespace mx {

constexpr int NB = LU_NB;  // columns per factorisation step

// ---- bandwidth and extraction ---------------------------------------------------------
__device__ inline int find_sub(const int64_t* offsets, int n_sub, int64_t q) {
  int lo = 0, hi = n_sub - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct ExtractArgs {
  int n_sub;
  int64_t sum_local;
  const int64_t* offsets;
  const int32_t* lists;
  const int32_t* inv_ptr;
  const int32_t* inv_pos;
  const int32_t* rowptr;
  const int32_t* col;
  const double* K;
  const double* M;
  double sr, si;  // s = k^2 + i xi_prec
  int32_t* band;  // [n_sub] (bandwidth pass)
  const int32_t* ld;
  const int64_t* moff;
  void* out;
  uint32_t* amax;  // [n_sub] largest |entry| written, as FP32 bits (write pass)
};

// modulus as FP32 bits: for non-negative floats the bit patterns order like the values, so
// an unsigned atomicMax over them takes the maximum in any arrival order
__device__ inline uint32_t abs_bits(float2 v) { return __float_as_uint(sqrtf(v.x * v.x + v.y * v.y)); }
__device__ inline uint32_t abs_bits(double2 v) { return __float_as_uint((float)sqrt(v.x * v.x + v.y * v.y)); }

template <typename T2, bool WRITE>
__global__ void k_extract(ExtractArgs a) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < a.sum_local;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int l = find_sub(a.offsets, a.n_sub, q);
    const int64_t lo = a.offsets[l], hi = a.offsets[l + 1];
    const int i = (int)(q - lo);
    const int32_t g = a.lists[q];
    int bmax = 0;
    int bw = 0;
    int ldl = 0;
    int64_t off = 0;
    uint32_t amax = 0;
    if (WRITE) { bw = a.band[l]; ldl = a.ld[l]; off = a.moff[l]; }
    for (int32_t e = a.rowptr[g]; e < a.rowptr[g + 1]; ++e) {
      const int32_t c = a.col[e];
      int j = -1;
      for (int32_t t = a.inv_ptr[c]; t < a.inv_ptr[c + 1]; ++t) {
        const int32_t p = a.inv_pos[t];
        if (p >= lo && p < hi) { j = (int)(p - lo); break; }
      }
      if (j < 0) continue;
      if (!WRITE) {
        bmax = max(bmax, abs(i - j));
      } else {
        const double re = a.K[e] - a.sr * a.M[e];
        const double im = -a.si * a.M[e];
        T2* A = reinterpret_cast<T2*>(a.out);
        const T2 v = conv<T2>(make_double2(re, im));
        A[bidx(off, ldl, bw, i, j)] = v;
        amax = max(amax, abs_bits(v));
      }
    }
    if (!WRITE) atomicMax(&a.band[l], bmax);
    else if (a.amax) atomicMax(a.amax + l, amax);
  }
}

// ---- batched band LU ----------------------------------------------------------------
// Status words: status[0] = number of zero / non-finite pivots met.
template <typename T2>
__global__ void k_lu_diag(BandBatch B, T2* A, int k0, int32_t* status) {
  __shared__ T2 s[NB][NB + 1];
  const int m = blockIdx.x;
  const int n = B.n[m], b = B.b[m], ld = B.ld[m];
  const int64_t off = B.off[m];
  if (k0 >= n) return;
  const int kb = min(NB, n - k0);
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int i = t % NB, j = t / NB;
    T2 v = czero<T2>();
    if (i < kb && j < kb && abs(i - j) <= b) v = A[bidx(off, ld, b, k0 + i, k0 + j)];
    s[i][j] = v;
  }
  __syncthreads();
  for (int k = 0; k < kb; ++k) {
    const T2 piv = s[k][k];
    const auto p2 = cabs2(piv);
    if (threadIdx.x == 0 && !(p2 > 0 && p2 < INFINITY)) atomicAdd(status, 1);
    const T2 inv = crcp(piv);
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < kb; i += blockDim.x) s[i][k] = cmul(s[i][k], inv);
    __syncthreads();
    const int w = kb - k - 1;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      const int i = k + 1 + t % w, j = k + 1 + t / w;
      T2 v = s[i][j];
      cfms(v, s[i][k], s[k][j]);
      s[i][j] = v;
    }
    __syncthreads();
  }
  uint32_t um = 0;
  for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) {
    const int i = t % kb, j = t / kb;
    if (abs(i - j) <= b) {
      A[bidx(off, ld, b, k0 + i, k0 + j)] = s[i][j];
      if (i <= j) um = max(um, abs_bits(s[i][j]));
    }
  }
  if (B.umax) {  // every thread of the block gets here (the early returns are block-uniform)
    um = __reduce_max_sync(0xffffffffu, um);
    if ((threadIdx.x & 31) == 0) atomicMax(B.umax + m, um);
  }
}

// Panels: rows below the block get L21 = A21 U11^{-1}; columns right of it get
// U12 = L11^{-1} A12. blockIdx.y < row chunks: rows; else columns.
template <typename T2>
__global__ void k_lu_panel(BandBatch B, T2* A, int k0) {
  __shared__ T2 s[NB][NB + 1];
  const int m = blockIdx.x;
  const int n = B.n[m], b = B.b[m], ld = B.ld[m];
  const int64_t off = B.off[m];
  if (k0 >= n) return;
  const int kb = min(NB, n - k0);
  const int k1 = k0 + kb;
  const int span = min(n, k1 + b) - k1;  // rows / columns within the band of the block
  if (span <= 0) return;
  const int chunks = (span + blockDim.x - 1) / blockDim.x;
  if ((int)blockIdx.y >= 2 * chunks) return;
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int i = t % NB, j = t / NB;
    T2 v = czero<T2>();
    if (i < kb && j < kb && abs(i - j) <= b) v = A[bidx(off, ld, b, k0 + i, k0 + j)];
    s[i][j] = v;
  }
  __syncthreads();
  const bool rows = (int)blockIdx.y < chunks;
  const int idx = ((rows ? blockIdx.y : blockIdx.y - chunks) * blockDim.x) + threadIdx.x;
  uint32_t um = 0;  // largest |U12| entry of this thread's column
  // loops fully unrolled over NB (entries k >= kb are zero and unused), so x stays in registers
  T2 x[NB];
  if (idx >= span) {
    // past the band: nothing to compute; stays for the block's growth reduction below
  } else if (rows) {
    const int i = k1 + idx;
#pragma unroll
    for (int k = 0; k < NB; ++k)
      x[k] = (k < kb && i - (k0 + k) <= b) ? A[bidx(off, ld, b, i, k0 + k)] : czero<T2>();
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
      if (k < kb && i - (k0 + k) <= b) A[bidx(off, ld, b, i, k0 + k)] = x[k];
  } else {
    const int j = k1 + idx;
#pragma unroll
    for (int k = 0; k < NB; ++k)
      x[k] = (k < kb && j - (k0 + k) <= b) ? A[bidx(off, ld, b, k0 + k, j)] : czero<T2>();
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
      if (k < kb && j - (k0 + k) <= b) {
        A[bidx(off, ld, b, k0 + k, j)] = x[k];
        um = max(um, abs_bits(x[k]));
      }
  }
  if (B.umax && !rows) {  // block-uniform branch: all 256 threads take part
    um = __reduce_max_sync(0xffffffffu, um);
    if ((threadIdx.x & 31) == 0 && um) atomicMax(B.umax + m, um);
  }
}

// Trailing update A22 -= L21 U12 over the band window, 64 x 64 tiles, 256 threads with
// 4 x 4 outputs each. blockIdx.y enumerates tiles of the (span x span) window.
template <typename T2>
__global__ void __launch_bounds__(256) k_lu_update(BandBatch B, T2* A, int k0) {
  __shared__ T2 sl[NB][64 + 1];
  __shared__ T2 su[NB][64 + 1];
  const int m = blockIdx.x;
  const int n = B.n[m], b = B.b[m], ld = B.ld[m];
  const int64_t off = B.off[m];
  if (k0 >= n) return;
  const int kb = min(NB, n - k0);
  const int k1 = k0 + kb;
  const int span = min(n, k1 + b) - k1;
  if (span <= 0) return;
  const int tiles = (span + 63) / 64;
  if ((int)blockIdx.y >= tiles * tiles) return;
  const int ti = blockIdx.y % tiles, tj = blockIdx.y / tiles;
  const int i0 = k1 + 64 * ti, j0 = k1 + 64 * tj;
  // skip tiles entirely outside the band
  if (i0 - (j0 + 63) > b || j0 - (i0 + 63) > b) return;
  for (int t = threadIdx.x; t < NB * 64; t += blockDim.x) {
    const int r = t % 64, k = t / 64;
    const int i = i0 + r, kk = k0 + k;
    sl[k][r] = (k < kb && i < n && i - kk <= b) ? A[bidx(off, ld, b, i, kk)] : czero<T2>();
    const int j = j0 + r;
    su[k][r] = (k < kb && j < n && j - kk <= b) ? A[bidx(off, ld, b, kk, j)] : czero<T2>();
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
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
      T2* p = A + bidx(off, ld, b, i, j);
      *p = csub(*p, acc[a][c]);
    }
  }
}

template <typename T2>
void band_lu(const BandBatch& B, T2* A, int max_n, int max_span, int32_t* status, cudaStream_t s,
             const int32_t* hn, const int32_t* hb, int kid_update, int tc_split) {
  const int chunks = (max_span + 255) / 256;
  const int tiles = (max_span + 63) / 64;
  const double esz = sizeof(T2);
  for (int k0 = 0; k0 < max_n; k0 += NB) {
    // algorithmic work of this step over the batch (complex MAC = 8 flops)
    double upd_flops = 0, upd_bytes = 0, pan_flops = 0, pan_bytes = 0;
    if (hn && hb)
      for (int m = 0; m < B.count; ++m) {
        if (k0 >= hn[m]) continue;
        const double kb = std::min(NB, hn[m] - k0);
        const double span = std::max(0, std::min(hn[m], k0 + (int)kb + hb[m]) - (k0 + (int)kb));
        upd_flops += 8.0 * span * span * kb;
        upd_bytes += esz * (2.0 * span * span + 2.0 * span * kb);
        pan_flops += 8.0 * span * kb * kb;
        pan_bytes += esz * 4.0 * span * kb;
      }
    {
      ProfScope ps(kid_update < 0 ? K_LU_DIAG : kid_update, s);
      MX_LAUNCH(k_lu_diag<T2><<<B.count, 256, 0, s>>>(B, A, k0, status));
      MX_CHECK_LAUNCH();
    }
    if (max_span > 0) {
      {
        ProfScope ps(kid_update < 0 ? K_LU_PANEL : kid_update, s, 1, pan_bytes, pan_flops);
        MX_LAUNCH(k_lu_panel<T2><<<dim3(B.count, 2 * chunks), 256, 0, s>>>(B, A, k0));
        MX_CHECK_LAUNCH();
      }
      ProfScope ps(kid_update < 0 ? K_LU_UPDATE : kid_update, s, 1, upd_bytes, upd_flops);
      if constexpr (std::is_same<T2, float2>::value) {
        if (tc_split > 0) {  // tcgen05 tensor-core update (TF32 or 3 x TF32)
          lu_update_tc(B, A, k0, max_span, tc_split, status + 2, s);
          continue;
        }
      }
      MX_LAUNCH(k_lu_update<T2><<<dim3(B.count, tiles * tiles), 256, 0, s>>>(B, A, k0));
      MX_CHECK_LAUNCH();
    }
  }
}

template void band_lu<double2>(const BandBatch&, double2*, int, int, int32_t*, cudaStream_t, const int32_t*,
                               const int32_t*, int, int);
template void band_lu<float2>(const BandBatch&, float2*, int, int, int32_t*, cudaStream_t, const int32_t*,
                              const int32_t*, int, int);

// ---- host: extraction and factorisation -------------------------------------------
static int round4(int x) { return (x + 3) & ~3; }

static ExtractArgs extract_args(const Problem& P) {
  ExtractArgs a{};
  a.n_sub = P.n_sub;
  a.sum_local = P.sum_local;
  a.offsets = P.offsets.p;
  a.lists = P.lists.p;
  a.inv_ptr = P.inv_ptr.p;
  a.inv_pos = P.inv_pos.p;
  a.rowptr = P.A.rowptr.p;
  a.col = P.A.col.p;
  a.K = P.A.K.p;
  a.M = P.A.M.p;
  a.sr = P.k * P.k;
  a.si = P.xi_prec;
  return a;
}

// Half-bandwidth of every minor (one pass over the CSR rows of all subdomains) and the
// band storage plan: h_band, h_ld, h_mat_off, band_entries.
void plan_local_storage(Problem& P) {
  cudaStream_t s = P.stream;
  ExtractArgs a = extract_args(P);
  DevBuf<int32_t> band(P.n_sub);
  MX_CUDA(cudaMemsetAsync(band.p, 0, band.bytes(), s));
  a.band = band.p;
  MX_LAUNCH(k_extract<float2, false><<<grid_for(P.sum_local, 256), 256, 0, s>>>(a));
  MX_CHECK_LAUNCH();
  P.h_band.assign(P.n_sub, 0);
  MX_CUDA(cudaMemcpyAsync(P.h_band.data(), band.p, band.bytes(), cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  P.h_ld.assign(P.n_sub, 0);
  P.h_mat_off.assign(P.n_sub + 1, 0);
  P.band_entries = 0;
  for (int l = 0; l < P.n_sub; ++l) {
    if (P.dense_local) P.h_band[l] = P.h_nl[l] - 1;
    const int64_t nn = P.h_nl[l], bb = std::min<int64_t>(P.h_band[l], nn - 1);
    P.band_entries += nn * (2 * bb + 1) - bb * (bb + 1);  // entries with |i - j| <= b
    P.h_ld[l] = round4(2 * P.h_band[l] + 1);
    P.h_mat_off[l + 1] = P.h_mat_off[l] + (int64_t)P.h_ld[l] * P.h_nl[l];
  }
}

// Device bytes the local factors (band + inverted diagonal blocks) will hold.
int64_t local_factor_bytes(Problem& P) {
  plan_local_storage(P);
  const int64_t esz = P.precision == MX_MIXED ? 8 : 16;
  int64_t blocks = 0;
  for (int l = 0; l < P.n_sub; ++l) blocks += (P.h_nl[l] + NB - 1) / NB;
  const int64_t panels = P.tune_local_tc ? panel_bytes_planned(P) : 0;
  // the explicit coarse inverse of the mixed form (the band factors of A^0 are smaller)
  const int64_t cinv =
      (P.coarse_m && P.precision == MX_MIXED && P.tune_coarse_inverse && P.coarse.n_dof <= COARSE_INVERSE_MAX)
          ? (int64_t)sizeof(float2) * P.coarse.n_dof * P.coarse.n_dof
          : 0;
  return esz * (P.h_mat_off[P.n_sub] + blocks * 2 * NB * NB) + panels + cinv;
}

void extract_minors(Problem& P) {
  cudaStream_t s = P.stream;
  const size_t esz = P.precision == MX_MIXED ? sizeof(float2) : sizeof(double2);
  plan_local_storage(P);
  ExtractArgs a{};
  a.n_sub = P.n_sub;
  a.sum_local = P.sum_local;
  a.offsets = P.offsets.p;
  a.lists = P.lists.p;
  a.inv_ptr = P.inv_ptr.p;
  a.inv_pos = P.inv_pos.p;
  a.rowptr = P.A.rowptr.p;
  a.col = P.A.col.p;
  a.K = P.A.K.p;
  a.M = P.A.M.p;
  a = extract_args(P);
  P.band.alloc(P.n_sub);
  P.ld.alloc(P.n_sub);
  P.mat_off.alloc(P.n_sub + 1);
  MX_CUDA(cudaMemcpyAsync(P.band.p, P.h_band.data(), P.n_sub * 4, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(P.ld.p, P.h_ld.data(), P.n_sub * 4, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(P.mat_off.p, P.h_mat_off.data(), (P.n_sub + 1) * 8, cudaMemcpyHostToDevice, s));
  const int64_t elems = P.h_mat_off[P.n_sub];
  P.factors.alloc(elems * esz);
  MX_CUDA(cudaMemsetAsync(P.factors.p, 0, P.factors.bytes(), s));
  a.band = P.band.p;
  a.ld = P.ld.p;
  a.moff = P.mat_off.p;
  a.out = P.factors.p;
  P.amax.alloc(P.n_sub);
  MX_CUDA(cudaMemsetAsync(P.amax.p, 0, P.amax.bytes(), s));
  a.amax = P.amax.p;
  if (P.bc == MX_BC_IMPEDANCE)
    extract_imp(P);  // ImpRAS: Galerkin matrices of the closed boxes, not minors of A
  else if (P.precision == MX_MIXED)
    MX_LAUNCH(k_extract<float2, true><<<grid_for(P.sum_local, 256), 256, 0, s>>>(a));
  else
    MX_LAUNCH(k_extract<double2, true><<<grid_for(P.sum_local, 256), 256, 0, s>>>(a));
  MX_CHECK_LAUNCH();
  MX_CUDA(cudaStreamSynchronize(s));
  P.minors_ready = true;
  P.factored = false;
}

// Inverses of the NB x NB diagonal blocks of L (unit lower) and U (upper) of every
// factored band matrix: block q of matrix m goes to Dinv + doff[m] + q * 2 NB^2 as two
// column-major NB x NB blocks [L_qq^{-1}, U_qq^{-1}] (zero outside the matrix). The sweeps
// then apply each diagonal block as a small matrix-vector product instead of a
// sequential substitution. One block per (matrix, diagonal block), thread j = column j.
template <typename T2>
__global__ void k_invert_diag(BandBatch B, const T2* A, const int64_t* doff, T2* Dinv) {
  __shared__ T2 L[NB][NB + 1], U[NB][NB + 1];
  const int m = blockIdx.x, q = blockIdx.y;
  const int n = B.n[m], b = B.b[m], ld = B.ld[m];
  const int64_t off = B.off[m];
  const int c0 = q * NB;
  if (c0 >= n) return;
  const int kb = min(NB, n - c0);
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int i = t % NB, k = t / NB;
    const bool in = i < kb && k < kb && abs(i - k) <= b;
    const T2 v = in ? A[bidx(off, ld, b, c0 + i, c0 + k)] : czero<T2>();
    L[i][k] = (i > k) ? v : czero<T2>();
    U[i][k] = (i <= k) ? v : czero<T2>();
  }
  __syncthreads();
  T2* out = Dinv + doff[m] + (int64_t)q * 2 * NB * NB;
  const int j = threadIdx.x;
  if (j < NB) {
    T2 x[NB];
    // L x = e_j (unit lower), forward
    for (int i = 0; i < NB; ++i) {
      T2 v = (i == j) ? mk(decltype(T2::x)(1), decltype(T2::x)(0)) : czero<T2>();
      for (int k = 0; k < i; ++k) cfms(v, L[i][k], x[k]);
      x[i] = (i < kb && j < kb) ? v : czero<T2>();
    }
    for (int i = 0; i < NB; ++i) out[(int64_t)j * NB + i] = x[i];
    // U x = e_j, backward
    for (int i = NB - 1; i >= 0; --i) {
      T2 v = (i == j) ? mk(decltype(T2::x)(1), decltype(T2::x)(0)) : czero<T2>();
      for (int k = i + 1; k < NB; ++k) cfms(v, U[i][k], x[k]);
      x[i] = (i < kb && j < kb) ? cmul(v, crcp(U[i][i])) : czero<T2>();
    }
    for (int i = 0; i < NB; ++i) out[NB * NB + (int64_t)j * NB + i] = x[i];
  }
}

template <typename T2>
void invert_diag_blocks(const BandBatch& B, const T2* A, const int64_t* doff, T2* Dinv, int max_n, cudaStream_t s) {
  const int nq = (max_n + NB - 1) / NB;
  ProfScope ps(K_LU_DIAG, s);
  MX_LAUNCH(k_invert_diag<T2><<<dim3(B.count, nq), 64, 0, s>>>(B, A, doff, Dinv));
  MX_CHECK_LAUNCH();
}
template void invert_diag_blocks<float2>(const BandBatch&, const float2*, const int64_t*, float2*, int, cudaStream_t);
template void invert_diag_blocks<double2>(const BandBatch&, const double2*, const int64_t*, double2*, int,
                                          cudaStream_t);

void factor_local(Problem& P) {
  factor_local_launch(P);
  factor_local_finish(P);
}

// queue the batched LU and the diagonal-block inversion (no host wait)
void factor_local_launch(Problem& P) {
  if (!P.minors_ready) extract_minors(P);
  P.umax.alloc(P.n_sub);
  MX_CUDA(cudaMemsetAsync(P.umax.p, 0, P.umax.bytes(), P.stream));
  BandBatch B{P.n_sub, P.nl.p, P.band.p, P.ld.p, P.mat_off.p, P.umax.p};
  int max_span = 0;
  for (int l = 0; l < P.n_sub; ++l) max_span = std::max(max_span, std::min(P.h_band[l], P.h_nl[l]));
  // offsets of the inverted diagonal blocks
  std::vector<int64_t> doff(P.n_sub + 1, 0);
  for (int l = 0; l < P.n_sub; ++l) doff[l + 1] = doff[l] + (int64_t)((P.h_nl[l] + NB - 1) / NB) * 2 * NB * NB;
  P.dinv_off.alloc(P.n_sub + 1);
  MX_CUDA(cudaMemcpyAsync(P.dinv_off.p, doff.data(), doff.size() * 8, cudaMemcpyHostToDevice, P.stream));
  const size_t esz = P.precision == MX_MIXED ? sizeof(float2) : sizeof(double2);
  P.dinv.alloc((size_t)doff[P.n_sub] * esz);
  if (P.precision == MX_MIXED && (P.tune_lu_tc == 0 || P.tune_lu_tc == 2) && band_lu_fused_fits(max_span)) {
    // one persistent launch, one CTA per subdomain, tensor-core trailing updates; booked with
    // every band entry read and written once and the flops of the blocked LU
    double flops = 0;
    for (int l = 0; l < P.n_sub; ++l)
      for (int k0 = 0; k0 < P.h_nl[l]; k0 += NB) {
        const double kb = std::min(NB, P.h_nl[l] - k0);
        const double span = std::max(0, std::min(P.h_nl[l] - k0 - (int)kb, P.h_band[l]));
        flops += 8.0 * span * span * kb + 8.0 * span * kb * kb + 8.0 / 3.0 * kb * kb * kb;
      }
    band_lu_fused(B, reinterpret_cast<float2*>(P.factors.p), P.dinv_off.p, reinterpret_cast<float2*>(P.dinv.p), 3,
                  P.tune_lu_grid, P.status.p, P.stream, 2.0 * sizeof(float2) * (double)P.band_entries, flops);
  } else if (P.precision == MX_MIXED) {
    band_lu<float2>(B, reinterpret_cast<float2*>(P.factors.p), P.max_local, max_span, P.status.p, P.stream,
                    P.h_nl.data(), P.h_band.data(), -1, P.tune_lu_tc == 4 ? 0 : P.tune_lu_tc);
    invert_diag_blocks<float2>(B, reinterpret_cast<float2*>(P.factors.p), P.dinv_off.p,
                               reinterpret_cast<float2*>(P.dinv.p), P.max_local, P.stream);
  } else {
    band_lu<double2>(B, reinterpret_cast<double2*>(P.factors.p), P.max_local, max_span, P.status.p, P.stream,
                     P.h_nl.data(), P.h_band.data(), -1, 0);
    invert_diag_blocks<double2>(B, reinterpret_cast<double2*>(P.factors.p), P.dinv_off.p,
                                reinterpret_cast<double2*>(P.dinv.p), P.max_local, P.stream);
  }
}

// wait for the queued factorisation, then the tensor-core panel images
void factor_local_finish(Problem& P) {
  MX_CUDA(cudaStreamSynchronize(P.stream));
  P.minors_ready = false;
  P.factored = true;
  P.panels.reset();
  P.panels_ok = false;
  if (P.precision == MX_MIXED && P.tune_local_tc) build_panels(P);
}

// ---- local solves -------------------------------------------------------------------
// One block per (subdomain, group of G right-hand sides). The window holds WIN rows of
// the right-hand side block (slot = row % WIN, WIN >= b + NB). Forward: unit lower L;
// backward: upper U. Rows leaving the forward window are the intermediate y, written to
// `out` and read back by the backward sweep, which overwrites them with z_l.
struct SolveArgs {
  int n_sub, nrhs;
  int64_t n_dof;
  const int64_t* offsets;  // positions of subdomain rows
  const int32_t* lists;
  const int32_t* nl;
  const int32_t* band;
  const int32_t* ld;
  const int64_t* moff;
  const void* factors;
  const void* dinv;       // inverted diagonal blocks
  const int64_t* doff;    // [n_sub] their offsets
  const void* v;  // [n][nrhs] c128 or c64 (right-hand side index fastest)
  int vtype;
  void* out;      // [sum_local][nrhs] of T2
  int win;        // window rows
  double alg_bytes, alg_flops;  // algorithmic traffic / work of one launch (profiling)
};

template <typename T2>
__device__ inline T2 load_v(const void* v, int vtype, int64_t idx) {
  if (vtype == 0) return conv<T2>(reinterpret_cast<const double2*>(v)[idx]);
  if (vtype == 3) {
    if constexpr (std::is_same<T2, float2>::value) {
      const float4 d = reinterpret_cast<const float4*>(v)[idx];
      return make_float2(d.x, d.y);
    } else {
      const float4 d = reinterpret_cast<const float4*>(v)[idx];
      return make_double2((double)d.x + (double)d.z, (double)d.y + (double)d.w);
    }
  }
  const float2 f = reinterpret_cast<const float2*>(v)[idx];
  return conv<T2>(make_double2(f.x, f.y));
}

// right-hand side entry (row, column): from v, or the identity for vtype 2
template <typename T2>
__device__ inline T2 rhs_value(const SolveArgs& a, int64_t row, int col) {
  if (a.vtype == 2) return row == col ? mk(decltype(T2::x)(1), decltype(T2::x)(0)) : czero<T2>();
  return load_v<T2>(a.v, a.vtype, row * a.nrhs + col);
}

// x_blk = D r_blk for the kb x kb diagonal block (D = L_qq^{-1}, unit lower, or
// D = U_qq^{-1}, upper; column-major NB x NB in global memory) on the window rows
// c0..c0+kb-1, all G right-hand sides. Every thread of the block takes part (256 threads).
template <typename T2, int G, bool UPPER>
__device__ inline void diag_apply(const T2* __restrict__ D, int c0, int kb, T2* W, int win, T2 (*Ds)[NB + 1]) {
  const int tid = threadIdx.x;
  for (int t = tid; t < NB * NB; t += 256) Ds[t % NB][t / NB] = D[t];
  __syncthreads();
  constexpr int PER = (NB * G + 255) / 256;
  const int s0 = c0 % win;
  T2 out[PER];
#pragma unroll
  for (int c = 0; c < PER; ++c) {
    const int t = tid + 256 * c;
    out[c] = czero<T2>();
    if (t < kb * G) {
      const int i = t / G, g = t % G;
      // D is zero outside its triangle and beyond kb; window slots always hold finite values
      if constexpr (std::is_same<T2, float2>::value) {
        CAcc2 s;
        cacc_zero(s);
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          int sk = s0 + k;
          if (sk >= win) sk -= win;
          cacc(s, Ds[i][k], W[sk * G + g]);
        }
        out[c] = cacc_value(s);
      } else {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          int sk = s0 + k;
          if (sk >= win) sk -= win;
          cfma(out[c], Ds[i][k], W[sk * G + g]);
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < PER; ++c) {
    const int t = tid + 256 * c;
    if (t < kb * G) W[((c0 + t / G) % win) * G + t % G] = out[c];
  }
  __syncthreads();
}

// W[i] -= sum_k F(i, k) W[k] over the block columns k in [c0, c0 + kb) ∩ [klo, khi) for one
// window row i and all G right-hand sides. Fixed 32-column trip count, factor entries
// loaded 16 at a time ahead of their use (out-of-range entries load as zero; window
// slots always hold finite values, so the extra products add exact zeros).
template <typename T2, int G>
__device__ __forceinline__ void row_update(const T2* __restrict__ F, int64_t off, int ld, int b, int i, int c0, int kb,
                                           int klo, int khi, T2* W, int win) {
  const int si = i % win, s0 = c0 % win;
  // chunk of factor entries in flight per thread: smaller for wide right-hand-side groups
  constexpr int CH = G >= 8 ? 8 : 16;
  if constexpr (std::is_same<T2, float2>::value) {
    // FP32: paired-FMA accumulation, two FFMA2 per complex product
    CAcc2 s[G];
#pragma unroll
    for (int g = 0; g < G; ++g) cacc_zero(s[g]);
#pragma unroll
    for (int kk = 0; kk < NB; kk += CH) {
      float2 l[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int k = c0 + kk + u;
        l[u] = (kk + u < kb && k >= klo && k < khi) ? F[bidx(off, ld, b, i, k)] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        int sk = s0 + kk + u;
        if (sk >= win) sk -= win;
#pragma unroll
        for (int g = 0; g < G; ++g) cacc(s[g], l[u], W[sk * G + g]);
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) W[si * G + g] = csub(W[si * G + g], cacc_value(s[g]));
    return;
  }
  T2 acc[G];
#pragma unroll
  for (int g = 0; g < G; ++g) acc[g] = W[si * G + g];
#pragma unroll
  for (int kk = 0; kk < NB; kk += CH) {
    T2 l[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int k = c0 + kk + u;
      l[u] = (kk + u < kb && k >= klo && k < khi) ? F[bidx(off, ld, b, i, k)] : czero<T2>();
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      int sk = s0 + kk + u;
      if (sk >= win) sk -= win;
#pragma unroll
      for (int g = 0; g < G; ++g) cfms(acc[g], l[u], W[sk * G + g]);
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) W[si * G + g] = acc[g];
}

template <typename T2, int G>
__global__ void __launch_bounds__(256, (sizeof(T2) == 8 && G < 16 ? 3 : 2)) k_local_solve(SolveArgs a) {
  extern __shared__ unsigned char smem_raw[];
  T2* W = reinterpret_cast<T2*>(smem_raw);  // [win][G]
  __shared__ T2 Ds[NB][NB + 1];             // diagonal block of the current step
  const int groups = (a.nrhs + G - 1) / G;
  const int l = blockIdx.x / groups;
  const int g0 = (blockIdx.x % groups) * G;
  const int gn = min(G, a.nrhs - g0);
  const int n = a.nl[l], b = a.band[l], ld = a.ld[l];
  const int64_t off = a.moff[l], pos0 = a.offsets[l];
  const T2* __restrict__ F = reinterpret_cast<const T2*>(a.factors);
  const T2* Dinv = reinterpret_cast<const T2*>(a.dinv);
  const int64_t doff = a.doff[l];
  T2* out = reinterpret_cast<T2*>(a.out);
  const int win = a.win;
  const int tid = threadIdx.x, nt = blockDim.x;

  // ---- forward sweep: L y = R^l v. Identity right-hand sides (vtype 2, columns g0..)
  // have y = 0 above row g0 (L is unit lower): the sweep starts at g0's block and writes
  // those zeros directly.
  const int cstart = a.vtype == 2 ? (g0 / NB) * NB : 0;
  for (int t = tid; t < cstart * G; t += nt) {
    const int i = t / G, g = t % G;
    if (g < gn) out[(pos0 + i) * a.nrhs + g0 + g] = czero<T2>();
  }
  for (int t = tid; t < win * G; t += nt) {
    const int i = cstart + t / G, g = t % G;
    W[(i % win) * G + g] = (i < n && g < gn) ? rhs_value<T2>(a, (int64_t)a.lists[pos0 + i], g0 + g) : czero<T2>();
  }
  __syncthreads();
  for (int c0 = cstart; c0 < n; c0 += NB) {
    const int c1 = min(c0 + NB, n);
    // diagonal block: x_blk = L_qq^{-1} r_blk with the precomputed inverse
    diag_apply<T2, G, false>(Dinv + doff + (int64_t)(c0 / NB) * 2 * NB * NB, c0, c1 - c0, W, win, Ds);
    // rows below the block within the band
    const int r1 = min(n, c1 + b);
    for (int i = c1 + tid; i < r1; i += nt) row_update<T2, G>(F, off, ld, b, i, c0, c1 - c0, max(c0, i - b), c1, W, win);
    __syncthreads();
    // retire rows c0..c1-1 (y), load rows entering the window
    for (int t = tid; t < (c1 - c0) * G; t += nt) {
      const int i = c0 + t / G, g = t % G;
      const T2 y = W[(i % win) * G + g];
      if (g < gn) out[(pos0 + i) * a.nrhs + g0 + g] = y;
      const int inew = i + win;
      if (inew < n) W[(inew % win) * G + g] = (g < gn) ? rhs_value<T2>(a, (int64_t)a.lists[pos0 + inew], g0 + g) : czero<T2>();
    }
    __syncthreads();
  }

  // ---- backward sweep: U z = y, blocks from the bottom. Identity right-hand sides form a
  // complex symmetric inverse: column j is needed only in rows >= j (the rest comes from
  // the transpose), so the sweep stops at g0's block; the rows above keep the zeros written
  // by the forward sweep until the caller mirrors the lower triangle.
  const int nblk = (n + NB - 1) / NB;
  const int bstop = cstart / NB;
  const int top0 = max(0, n - win);
  for (int t = tid; t < (n - top0) * G; t += nt) {
    const int i = top0 + t / G, g = t % G;
    W[(i % win) * G + g] = (g < gn) ? out[(pos0 + i) * a.nrhs + g0 + g] : czero<T2>();
  }
  __syncthreads();
  for (int blk = nblk - 1; blk >= bstop; --blk) {
    const int c0 = blk * NB, c1 = min(c0 + NB, n);
    // diagonal block: x_blk = U_qq^{-1} r_blk with the precomputed inverse
    diag_apply<T2, G, true>(Dinv + doff + (int64_t)(c0 / NB) * 2 * NB * NB + NB * NB, c0, c1 - c0, W, win, Ds);
    // rows above the block within the band
    const int r0 = max(0, c0 - b);
    for (int i = r0 + tid; i < c0; i += nt) row_update<T2, G>(F, off, ld, b, i, c0, c1 - c0, c0, min(c1, i + b + 1), W, win);
    __syncthreads();
    for (int t = tid; t < (c1 - c0) * G; t += nt) {
      const int i = c0 + t / G, g = t % G;
      if (g < gn) out[(pos0 + i) * a.nrhs + g0 + g] = W[(i % win) * G + g];
      const int inew = i - win;
      if (inew >= 0)
        W[(inew % win) * G + g] = (g < gn) ? out[(pos0 + inew) * a.nrhs + g0 + g] : czero<T2>();
    }
    __syncthreads();
  }
}

template <typename T2, int G>
static void launch_local_solve(const SolveArgs& a, int win, cudaStream_t s, int kid = K_LOCAL_SOLVE) {
  const size_t smem = (size_t)win * G * sizeof(T2);
  // dynamic window + the static diagonal-block tile must fit the 227 KB per-block limit
  MX_REQUIRE(smem + sizeof(T2) * NB * (NB + 1) <= 227 * 1024, MX_EINVAL, "local solve window exceeds shared memory");
  static size_t configured = 0;
  if (smem > configured) {
    MX_CUDA(cudaFuncSetAttribute(k_local_solve<T2, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = smem;
  }
  const int groups = (a.nrhs + G - 1) / G;
  ProfScope ps(kid, s, 1, a.alg_bytes, a.alg_flops);
  MX_LAUNCH(k_local_solve<T2, G><<<a.n_sub * groups, 256, smem, s>>>(a));
  MX_CHECK_LAUNCH();
}

// X[i][j] = X[j][i] for i < j (row-major n x n): fills the upper triangle of a complex
// symmetric matrix from its lower triangle, 32 x 32 tiles staged in shared memory
__global__ void k_mirror_lower(int n, float2* X) {
  __shared__ float2 t[32][33];
  const int ti = blockIdx.y, tj = blockIdx.x;  // target tile (rows ti, columns tj), ti <= tj
  if (ti > tj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {  // source tile (rows tj, columns ti), coalesced along ti
    const int i = tj * 32 + r, j = ti * 32 + tx;
    if (i < n && j < n) t[r][tx] = X[(int64_t)i * n + j];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = ti * 32 + r, j = tj * 32 + tx;
    if (i < n && j < n && i < j) X[(int64_t)i * n + j] = t[tx][r];
  }
}

__global__ void k_iota(int n, int32_t* p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

// X = (A^0)^{-1} (c64, row-major n_c x n_c) from the c64 band factors of the coarse
// matrix: the band sweeps of the local solves on the identity columns, G at a time.
void coarse_inverse(Problem& P, float2* X) {
  const int nc = (int)P.n_c, b = P.coarse_band;
  cudaStream_t s = P.stream;
  DevBuf<int64_t> offs(2), moff(1), doff(1);
  DevBuf<int32_t> lists(nc), nl(1), band(1), ld(1);
  const int64_t h_offs[2] = {0, nc}, zero = 0;
  const int32_t h_nl = nc, h_b = b, h_ld = (int32_t)P.ld_c;
  MX_CUDA(cudaMemcpyAsync(offs.p, h_offs, 16, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(moff.p, &zero, 8, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(doff.p, &zero, 8, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(nl.p, &h_nl, 4, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(band.p, &h_b, 4, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(ld.p, &h_ld, 4, cudaMemcpyHostToDevice, s));
  MX_LAUNCH(k_iota<<<grid_for(nc, 256), 256, 0, s>>>(nc, lists.p));
  MX_CHECK_LAUNCH();
  SolveArgs a{};
  a.n_sub = 1;
  a.nrhs = nc;
  a.n_dof = nc;
  a.offsets = offs.p;
  a.lists = lists.p;
  a.nl = nl.p;
  a.band = band.p;
  a.ld = ld.p;
  a.moff = moff.p;
  a.factors = P.A0f.p;
  a.dinv = P.c_dinvf.p;
  a.doff = doff.p;
  a.v = nullptr;
  a.vtype = 2;
  a.out = X;
  a.win = std::max(NB, std::min(nc, b + NB));
  MX_REQUIRE((size_t)a.win * 8 * sizeof(float2) <= 200 * 1024, MX_EINVAL, "coarse bandwidth too large for the inverse");
  const double entries = (double)nc * (2.0 * b + 1.0) - (double)b * (b + 1.0);
  a.alg_bytes = 8.0 * entries + 8.0 * (double)nc * nc;
  a.alg_flops = 4.0 * entries * nc;  // each sweep covers about half of the columns' rows
  if ((size_t)a.win * 16 * sizeof(float2) <= 100 * 1024) launch_local_solve<float2, 16>(a, a.win, s, K_COARSE_INV);
  else launch_local_solve<float2, 8>(a, a.win, s, K_COARSE_INV);
  {
    ProfScope ps(K_COARSE_INV, s, 1, 16.0 * (double)nc * nc, 0.0);
    const unsigned tl = (unsigned)((nc + 31) / 32);
    MX_LAUNCH(k_mirror_lower<<<dim3(tl, tl), dim3(32, 8), 0, s>>>((int)nc, X));
    MX_CHECK_LAUNCH();
  }
  MX_CUDA(cudaStreamSynchronize(s));
}

void local_solves(Problem& P, const void* v, int vtype, void* loc, int nrhs) {
  MX_REQUIRE(P.factored, MX_ENOTFACTORED, "local solves before factor");
  SolveArgs a{};
  a.n_sub = P.n_sub;
  a.nrhs = nrhs;
  a.n_dof = P.fine.n_dof;
  a.offsets = P.offsets.p;
  a.lists = P.lists.p;
  a.nl = P.nl.p;
  a.band = P.band.p;
  a.ld = P.ld.p;
  a.moff = P.mat_off.p;
  a.factors = P.factors.p;
  a.dinv = P.dinv.p;
  a.doff = P.dinv_off.p;
  a.v = v;
  a.vtype = vtype;
  a.out = loc;
  int bmax = 0;
  for (int l = 0; l < P.n_sub; ++l) bmax = std::max(bmax, std::min(P.h_band[l], P.h_nl[l]));
  // window rows: at least one block of NB (the slot arithmetic in row_update / diag_apply
  // wraps once, so it needs win >= NB), at most the largest subdomain or band + block
  a.win = std::max(NB, std::min(P.max_local, bmax + NB));
  MX_REQUIRE(a.win >= NB, MX_EINVAL, "local solve window smaller than one block");
  {
    const double esz = P.precision == MX_MIXED ? 8.0 : 16.0;
    // factors read once, right-hand sides gathered once (c128), solutions written once
    a.alg_bytes = esz * (double)P.band_entries + (16.0 + esz) * (double)P.sum_local * nrhs;
    a.alg_flops = 8.0 * (double)P.band_entries * nrhs;
  }
  const bool mixed = P.precision == MX_MIXED;
  if (mixed && P.tune_local_tc) {
    if (!P.panels_ok) build_panels(P);
    if (P.panels_ok) {
      local_solves_tc(P, v, vtype, loc, nrhs, a.alg_bytes, a.alg_flops);
      return;
    }
  }
  // right-hand sides per block: the window must fit in shared memory
  const size_t esz = mixed ? 8 : 16;
  int G = 1;
  const int gmax = P.tune_local_group > 0 ? std::min(16, P.tune_local_group) : 16;
  while (G < nrhs && G < gmax) G *= 2;
  while (G > 1 && (size_t)a.win * G * esz > 100 * 1024) G /= 2;
  MX_REQUIRE((size_t)a.win * esz <= 200 * 1024, MX_EINVAL, "subdomain bandwidth too large for the local solve window");
  if (mixed) {
    switch (G) {
      case 16: launch_local_solve<float2, 16>(a, a.win, P.stream); break;
      case 8: launch_local_solve<float2, 8>(a, a.win, P.stream); break;
      case 4: launch_local_solve<float2, 4>(a, a.win, P.stream); break;
      case 2: launch_local_solve<float2, 2>(a, a.win, P.stream); break;
      default: launch_local_solve<float2, 1>(a, a.win, P.stream); break;
    }
  } else {
    switch (G) {
      case 16: launch_local_solve<double2, 16>(a, a.win, P.stream); break;
      case 8: launch_local_solve<double2, 8>(a, a.win, P.stream); break;
      case 4: launch_local_solve<double2, 4>(a, a.win, P.stream); break;
      case 2: launch_local_solve<double2, 2>(a, a.win, P.stream); break;
      default: launch_local_solve<double2, 1>(a, a.win, P.stream); break;
    }
  }
}

}  // namespace mx

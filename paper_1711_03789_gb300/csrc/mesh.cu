// Mesh and DOF generation (Sec. 2.2) and subdomain index sets (Sec. 3.1, Eq. 3.1).
//
// The unit cube has n^3 cubes; cube c = (i, j, l) holds 6 Kuhn tetrahedra, one per
// permutation s of the axes (lexicographic order), with vertex path
// c, c + e_s0, c + e_s0 + e_s1, c + (1,1,1). Every mesh edge is (v, v + D_d) for one of
// the 7 directions D (3 axes, 3 face diagonals, the body diagonal), oriented from the
// lower to the higher vertex id. Edges on a boundary face carry no DOF (PEC, Eq. 1.4);
// the others are numbered in increasing key 7 v + d. With the impedance condition (Eq. imp)
// every edge is a DOF, and the subdomains are closed boxes (ImpRAS, Sec. 6.3).
#include "problem.cuh"

namespace mx {

__constant__ int c_dirs[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                                 {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
__constant__ int c_perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
__constant__ int c_ledge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
// direction index of the 0/1 step vector encoded as dx + 2 dy + 4 dz
__constant__ int c_dir_of_code[8] = {-1, 0, 1, 3, 2, 4, 5, 6};

__global__ void k_edge_flags(int n, int all_edges, int32_t* flag) {
  const int64_t total = (int64_t)(n + 1) * (n + 1) * (n + 1) * 7;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / 7;
    const int d = (int)(t % 7);
    const int c[3] = {(int)(v % (n + 1)), (int)((v / (n + 1)) % (n + 1)), (int)(v / ((int64_t)(n + 1) * (n + 1)))};
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      const int D = c_dirs[d][a];
      if (c[a] + D > n) ok = false;                   // edge leaves the grid
      if (!all_edges && D == 0 && (c[a] == 0 || c[a] == n)) ok = false;  // lies on a boundary face
    }
    flag[t] = ok ? 1 : 0;
  }
}

__global__ void k_edge_numbers(int64_t total, const int32_t* flag, const int32_t* pre,
                               int32_t* edge_dof, int32_t* dof_key) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (flag[t]) {
      edge_dof[t] = pre[t];
      dof_key[pre[t]] = (int32_t)t;
    } else {
      edge_dof[t] = -1;
    }
  }
}

__global__ void k_tet2dof(int n, const int32_t* edge_dof, int32_t* tet2dof) {
  const int64_t ntet = 6LL * n * n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntet;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cube = t / 6;
    const int p = (int)(t % 6);
    int P[4][3];
    P[0][0] = (int)(cube % n);
    P[0][1] = (int)((cube / n) % n);
    P[0][2] = (int)(cube / ((int64_t)n * n));
    for (int k = 0; k < 3; ++k) {
      for (int a = 0; a < 3; ++a) P[k + 1][a] = P[k][a];
      P[k + 1][c_perms[p][k]] += 1;
    }
    for (int e = 0; e < 6; ++e) {
      const int a = c_ledge[e][0], b = c_ledge[e][1];
      const int code = (P[b][0] - P[a][0]) + 2 * (P[b][1] - P[a][1]) + 4 * (P[b][2] - P[a][2]);
      const int64_t v = P[a][0] + (int64_t)(n + 1) * (P[a][1] + (int64_t)(n + 1) * P[a][2]);
      tet2dof[t * 6 + e] = edge_dof[v * 7 + c_dir_of_code[code]];
    }
  }
}

void build_mesh(MeshDev& m, int n, cudaStream_t s, bool all_edges) {
  m.n = n;
  const int64_t total = (int64_t)(n + 1) * (n + 1) * (n + 1) * 7;
  MX_REQUIRE(total < (1LL << 31), MX_EINVAL, "mesh too large for 32-bit edge keys");
  DevBuf<int32_t> flag(total), pre(total + 1);
  MX_LAUNCH(k_edge_flags<<<grid_for(total, 256), 256, 0, s>>>(n, all_edges ? 1 : 0, flag.p));
  MX_CHECK_LAUNCH();
  m.n_dof = exclusive_scan_i32(flag.p, pre.p, total, s);
  m.edge_dof.alloc(total);
  m.dof_key.alloc(std::max<int64_t>(m.n_dof, 1));
  MX_LAUNCH(k_edge_numbers<<<grid_for(total, 256), 256, 0, s>>>(total, flag.p, pre.p, m.edge_dof.p, m.dof_key.p));
  MX_CHECK_LAUNCH();
  const int64_t ntet = 6LL * n * n * n;
  m.tet2dof.alloc(ntet * 6);
  MX_LAUNCH(k_tet2dof<<<grid_for(ntet, 256), 256, 0, s>>>(n, m.edge_dof.p, m.tet2dof.p));
  MX_CHECK_LAUNCH();
  MX_CUDA(cudaStreamSynchronize(s));
}

// ---- subdomains ---------------------------------------------------------------------
// box i along an axis: cells [core i, min(core (i+1), n)) widened by `overlap`, clipped
static inline void span(int n, int core, int overlap, int i, int& lo, int& hi) {
  lo = std::max(core * i - overlap, 0);
  hi = std::min(std::min(core * (i + 1), n) + overlap, n);
}

// Edges with both ends in the box [lo, hi] (vertex indices) that do not lie on a box face;
// closed: all edges of the box, per direction D the product over axes of (len + 1 - D).
static inline int64_t box_count(int a, int b, int c, bool closed) {
  if (closed) {
    static const int D[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
    int64_t t = 0;
    for (int d = 0; d < 7; ++d) t += (int64_t)(a + 1 - D[d][0]) * (b + 1 - D[d][1]) * (c + 1 - D[d][2]);
    return t;
  }
  return (int64_t)a * (b - 1) * (c - 1) + (int64_t)b * (a - 1) * (c - 1) + (int64_t)c * (a - 1) * (b - 1) +
         (int64_t)a * b * (c - 1) + (int64_t)a * c * (b - 1) + (int64_t)b * c * (a - 1) + (int64_t)a * b * c;
}

struct BoxArgs {
  int n;
  int closed;  // keep the edges on the box faces
  const int32_t* box;  // [n_sub][6]
  const int64_t* offsets;
  const int32_t* edge_dof;
  int32_t* lists;
};

// One block per subdomain: candidates (local vertex in z, y, x order, then direction)
// are visited in increasing key order and compacted in order, so each list is sorted.
__global__ void k_box_lists(BoxArgs a) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t running;
  const int l = blockIdx.x;
  const int32_t* B = a.box + 6 * l;
  const int nvx = B[3] - B[0] + 1, nvy = B[4] - B[1] + 1, nvz = B[5] - B[2] + 1;
  const int64_t total = (int64_t)nvx * nvy * nvz * 7;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t base = 0; base < total; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    int take = 0;
    int32_t dof = -1;
    if (t < total) {
      const int d = (int)(t % 7);
      const int64_t lv = t / 7;
      const int c[3] = {B[0] + (int)(lv % nvx), B[1] + (int)((lv / nvx) % nvy), B[2] + (int)(lv / ((int64_t)nvx * nvy))};
      bool ok = true;
      for (int ax = 0; ax < 3; ++ax) {
        const int D = c_dirs[d][ax];
        if (c[ax] + D > B[3 + ax]) ok = false;
        if (!a.closed && D == 0 && (c[ax] == B[ax] || c[ax] == B[3 + ax])) ok = false;
      }
      if (ok) {
        const int64_t v = c[0] + (int64_t)(a.n + 1) * (c[1] + (int64_t)(a.n + 1) * c[2]);
        dof = a.edge_dof[v * 7 + d];
        take = dof >= 0;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, take);
    const int within = __popc(m & ((1u << lane) - 1));
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += warp_tot[w];
      all += warp_tot[w];
    }
    const int64_t at = running + before + within;
    if (take && at < a.offsets[l + 1] - a.offsets[l]) a.lists[a.offsets[l] + at] = dof;
    __syncthreads();
    if (threadIdx.x == 0) running += all;
    __syncthreads();
  }
}

struct InvArgs {
  int n, core, overlap, N, closed;
  int64_t n_dof;
  const int32_t* dof_key;
  const int32_t* box;
  const int64_t* offsets;
  const int32_t* nl;
  const int32_t* lists;
  int32_t* count;  // count pass
  const int32_t* ptr;  // fill pass
  int32_t* pos;
};

// Candidate boxes along one axis for an edge starting at coordinate c with step D.
__device__ inline int axis_boxes(int c, int D, int n, int core, int overlap, int N, int closed, int* out) {
  int k = 0;
  const int i0 = max(0, (c - overlap) / core - 1), i1 = min(N - 1, (c + overlap) / core + 1);
  for (int i = i0; i <= i1; ++i) {
    const int lo = max(core * i - overlap, 0);
    const int hi = min(min(core * (i + 1), n) + overlap, n);
    if (c < lo || c + D > hi) continue;
    if (!closed && D == 0 && (c == lo || c == hi)) continue;
    out[k++] = i;
  }
  return k;
}

template <bool FILL>
__global__ void k_inverse_map(InvArgs a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n_dof;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t key = a.dof_key[i];
    const int d = key % 7;
    const int64_t v = key / 7;
    const int c[3] = {(int)(v % (a.n + 1)), (int)((v / (a.n + 1)) % (a.n + 1)), (int)(v / ((int64_t)(a.n + 1) * (a.n + 1)))};
    int bx[16], by[16], bz[16];
    const int nx = axis_boxes(c[0], c_dirs[d][0], a.n, a.core, a.overlap, a.N, a.closed, bx);
    const int ny = axis_boxes(c[1], c_dirs[d][1], a.n, a.core, a.overlap, a.N, a.closed, by);
    const int nz = axis_boxes(c[2], c_dirs[d][2], a.n, a.core, a.overlap, a.N, a.closed, bz);
    if (!FILL) {
      a.count[i] = nx * ny * nz;
      continue;
    }
    int w = a.ptr[i];
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const int l = bx[x] + a.N * (by[y] + a.N * bz[z]);
          const int32_t* L = a.lists + a.offsets[l];
          int lo = 0, hi = a.nl[l] - 1, at = -1;
          while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int32_t val = L[mid];
            if (val == (int32_t)i) { at = mid; break; }
            if (val < (int32_t)i) lo = mid + 1; else hi = mid - 1;
          }
          a.pos[w++] = (at >= 0) ? (int32_t)(a.offsets[l] + at) : -1;
        }
  }
}

// Owner of every DOF for the restricted variants (Sec. 6.3): the core box holding the
// edge midpoint (twice the midpoint is 2c + D in vertex units), and the position of the DOF
// in the owner's list (-1 if the owner does not hold it, which overlap >= 1 rules out).
__global__ void k_owner_pos(int n, int core, int N, int64_t n_dof, const int32_t* dof_key, const int64_t* offsets,
                            const int32_t* nl, const int32_t* lists, int32_t* own_pos, int32_t* missing) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_dof; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t key = dof_key[i];
    const int d = key % 7;
    const int64_t v = key / 7;
    const int c[3] = {(int)(v % (n + 1)), (int)((v / (n + 1)) % (n + 1)), (int)(v / ((int64_t)(n + 1) * (n + 1)))};
    int b[3];
    for (int ax = 0; ax < 3; ++ax) b[ax] = min((2 * c[ax] + c_dirs[d][ax]) / (2 * core), N - 1);
    const int l = b[0] + N * (b[1] + N * b[2]);
    const int32_t* L = lists + offsets[l];
    int lo = 0, hi = nl[l] - 1, at = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int32_t val = L[mid];
      if (val == (int32_t)i) { at = mid; break; }
      if (val < (int32_t)i) lo = mid + 1; else hi = mid - 1;
    }
    own_pos[i] = at >= 0 ? (int32_t)(offsets[l] + at) : -1;
    if (at < 0) atomicAdd(missing, 1);
  }
}

void build_owner(Problem& P) {
  if (P.own_pos.p) return;
  MX_REQUIRE(P.overlap >= 1, MX_EINVAL, "the restricted variants need an overlap of at least one cell");
  cudaStream_t s = P.stream;
  const int64_t nd = P.fine.n_dof;
  DevBuf<int32_t> own(nd), missing(1);
  MX_CUDA(cudaMemsetAsync(missing.p, 0, 4, s));
  MX_LAUNCH(k_owner_pos<<<grid_for(nd, 256), 256, 0, s>>>(P.n, P.core, P.n_per_axis, nd, P.fine.dof_key.p, P.offsets.p,
                                                         P.nl.p, P.lists.p, own.p, missing.p));
  MX_CHECK_LAUNCH();
  int32_t h_missing = 0;
  MX_CUDA(cudaMemcpyAsync(&h_missing, missing.p, 4, cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  MX_REQUIRE(h_missing == 0, MX_EINVAL, "a DOF is not held by the subdomain that owns it");
  P.own_pos = std::move(own);
}

void build_subdomains(Problem& P) {
  cudaStream_t s = P.stream;
  const int n = P.n;
  const int N = (n + P.core - 1) / P.core;
  const bool closed = P.bc == MX_BC_IMPEDANCE;
  P.n_per_axis = N;
  P.n_sub = N * N * N;
  P.box.assign((size_t)P.n_sub * 6, 0);
  P.h_offsets.assign(P.n_sub + 1, 0);
  P.h_nl.assign(P.n_sub, 0);
  P.max_local = 0;
  for (int iz = 0; iz < N; ++iz)
    for (int iy = 0; iy < N; ++iy)
      for (int ix = 0; ix < N; ++ix) {
        const int l = ix + N * (iy + N * iz);
        int* B = &P.box[6 * l];
        span(n, P.core, P.overlap, ix, B[0], B[3]);
        span(n, P.core, P.overlap, iy, B[1], B[4]);
        span(n, P.core, P.overlap, iz, B[2], B[5]);
        const int64_t cnt = box_count(B[3] - B[0], B[4] - B[1], B[5] - B[2], closed);
        MX_REQUIRE(cnt > 0, MX_EINVAL, "a subdomain has no interior edge (core/overlap too small)");
        P.h_nl[l] = (int32_t)cnt;
        P.max_local = std::max<int>(P.max_local, (int)cnt);
      }
  for (int l = 0; l < P.n_sub; ++l) P.h_offsets[l + 1] = P.h_offsets[l] + P.h_nl[l];
  P.sum_local = P.h_offsets[P.n_sub];
  DevBuf<int32_t> dbox(P.box.size());
  P.offsets.alloc(P.n_sub + 1);
  P.nl.alloc(P.n_sub);
  P.lists.alloc(P.sum_local);
  MX_CUDA(cudaMemcpyAsync(dbox.p, P.box.data(), P.box.size() * 4, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(P.offsets.p, P.h_offsets.data(), (P.n_sub + 1) * 8, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(P.nl.p, P.h_nl.data(), P.n_sub * 4, cudaMemcpyHostToDevice, s));
  BoxArgs ba{n, closed ? 1 : 0, dbox.p, P.offsets.p, P.fine.edge_dof.p, P.lists.p};
  MX_LAUNCH(k_box_lists<<<P.n_sub, 256, 0, s>>>(ba));
  MX_CHECK_LAUNCH();

  const int64_t nd = P.fine.n_dof;
  DevBuf<int32_t> cnt(nd);
  P.inv_ptr.alloc(nd + 1);
  InvArgs ia{n, P.core, P.overlap, N, closed ? 1 : 0, nd, P.fine.dof_key.p, dbox.p, P.offsets.p, P.nl.p,
             P.lists.p, cnt.p, nullptr, nullptr};
  MX_LAUNCH(k_inverse_map<false><<<grid_for(nd, 256), 256, 0, s>>>(ia));
  MX_CHECK_LAUNCH();
  const int64_t total = exclusive_scan_i32(cnt.p, P.inv_ptr.p, nd, s);
  MX_REQUIRE(total == P.sum_local, MX_EINVAL, "subdomain cover mismatch");
  P.inv_pos.alloc(P.sum_local);
  ia.ptr = P.inv_ptr.p;
  ia.pos = P.inv_pos.p;
  MX_LAUNCH(k_inverse_map<true><<<grid_for(nd, 256), 256, 0, s>>>(ia));
  MX_CHECK_LAUNCH();
  MX_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mx

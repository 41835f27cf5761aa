// Assembly of the curl-curl and mass matrices (Eq. 2.2, Sec. 2.2), the load vector and
// the coarse restriction R^0 (Eq. 3.2).
//
// Whitney basis of the oriented edge (p -> q): w_pq = lam_p grad lam_q - lam_q grad lam_p,
// curl w_pq = 2 grad lam_p x grad lam_q. On the Kuhn tetrahedron of permutation s with
// cell size h the barycentric gradients are g/h with the integer vectors
//   g0 = -e_s0, g1 = e_s0 - e_s1, g2 = e_s1 - e_s2, g3 = e_s2,   |T| = h^3 / 6,
// and int lam_i lam_j = |T| (1 + delta_ij) / 20. Hence every element entry is an integer
// times one scale:
//   K_e[(pq),(rs)] = (2 / (3h)) (g_p x g_q).(g_r x g_s)
//   M_e[(pq),(rs)] = (h / 120) [ (g_q.g_s)(1+d_pr) - (g_q.g_r)(1+d_ps)
//                                - (g_p.g_s)(1+d_qr) + (g_p.g_r)(1+d_qs) ].
// Rows are assembled by gathering over the tetrahedra around each edge in a fixed order
// (no atomics), the integer parts are summed exactly and scaled once, so K and M are
// deterministic and exact up to that single rounding.
//
// Impedance condition (Eq. imp): B_ij = int_{boundary} (w_j)_T . (w_i)_T over the boundary
// triangles. On a triangle in a plane normal to axis a the tangential trace of w_pq is the
// triangle's Whitney form with the surface gradients g_i / h with their a-components
// dropped, int_F lam_i lam_j = |F| (1 + delta_ij) / 12 and |F| = h^2 / 2, so
//   B_F[(pq),(rs)] = (1 / 24) [ same bracket as M_e with the projected g ],
// independent of h. The same row gather restricted to a box (tetrahedra inside it,
// triangles on its surface) gives the ImpRAS local matrices (Sec. 6.3).
#include "df64.cuh"
#include "problem.cuh"

namespace mx {

__constant__ int a_dirs[7][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                                 {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};
__constant__ int a_perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
__constant__ int a_ledge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
__constant__ int a_dir_of_code[8] = {-1, 0, 1, 3, 2, 4, 5, 6};

// Integer gradient vectors g[4][3] of the Kuhn tetrahedron of permutation p.
__device__ inline void kuhn_grads(int p, int g[4][3]) {
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 3; ++a) g[i][a] = 0;
  const int s0 = a_perms[p][0], s1 = a_perms[p][1], s2 = a_perms[p][2];
  g[0][s0] = -1;
  g[1][s0] = 1; g[1][s1] -= 1;
  g[2][s1] = 1; g[2][s2] -= 1;
  g[3][s2] = 1;
}

__device__ inline int idot(const int* a, const int* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ inline void icross(const int* a, const int* b, int* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ inline void elem_int(int p, int ea, int eb, int& ik, int& im) {
  int g[4][3];
  kuhn_grads(p, g);
  const int P = a_ledge[ea][0], Q = a_ledge[ea][1], R = a_ledge[eb][0], S = a_ledge[eb][1];
  int c1[3], c2[3];
  icross(g[P], g[Q], c1);
  icross(g[R], g[S], c2);
  ik = idot(c1, c2);
  im = idot(g[Q], g[S]) * (1 + (P == R)) - idot(g[Q], g[R]) * (1 + (P == S)) -
       idot(g[P], g[S]) * (1 + (Q == R)) + idot(g[P], g[R]) * (1 + (Q == S));
}

// Path vertex index (0..3) of the 0/1 corner vector q in the Kuhn path of permutation p,
// or -1 if the corner is not on the path.
__device__ inline int path_index(int p, const int* q) {
  const int k = q[0] + q[1] + q[2];
  for (int i = 0; i < k; ++i)
    if (!q[a_perms[p][i]]) return -1;
  return k;
}

__device__ inline int ledge_index(int a, int b) {
  // (0,1)->0 (0,2)->1 (0,3)->2 (1,2)->3 (1,3)->4 (2,3)->5
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// Boundary-mass integer of local edges ea, eb on a tetrahedron face normal to axis ax.
__device__ inline int face_int(int p, int ea, int eb, int ax) {
  int g[4][3];
  kuhn_grads(p, g);
  for (int i = 0; i < 4; ++i) g[i][ax] = 0;
  const int P = a_ledge[ea][0], Q = a_ledge[ea][1], R = a_ledge[eb][0], S = a_ledge[eb][1];
  return idot(g[Q], g[S]) * (1 + (P == R)) - idot(g[Q], g[R]) * (1 + (P == S)) -
         idot(g[P], g[S]) * (1 + (Q == R)) + idot(g[P], g[R]) * (1 + (Q == S));
}

// Tetrahedra containing the edge from vertex c (grid coords) with direction d whose cube
// lies in the box of vertices [blo, bhi], in a fixed order (cubes in z, y, x order of their
// corner offsets, then permutations). Writes tet ids and the local edge index of the edge
// in each. Returns the count (<= 6).
__device__ inline int edge_tets(int n, const int* c, int d, int64_t* tets, int* loc, const int* blo,
                                const int* bhi) {
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    if (a_dirs[d][a]) { lo[a] = c[a]; hi[a] = c[a]; }
    else { lo[a] = max(c[a] - 1, blo[a]); hi[a] = min(c[a], bhi[a] - 1); }
  }
  int k = 0;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int q0[3] = {c[0] - x, c[1] - y, c[2] - z};
        const int q1[3] = {q0[0] + a_dirs[d][0], q0[1] + a_dirs[d][1], q0[2] + a_dirs[d][2]};
        const int64_t cube = x + (int64_t)n * (y + (int64_t)n * z);
        for (int p = 0; p < 6; ++p) {
          const int ia = path_index(p, q0), ib = path_index(p, q1);
          if (ia < 0 || ib < 0) continue;
          tets[k] = cube * 6 + p;
          loc[k] = ledge_index(ia, ib);
          ++k;
        }
      }
  return k;
}

__device__ inline void key_to_coords(int32_t key, int n, int* c, int& d) {
  d = key % 7;
  const int64_t v = key / 7;
  c[0] = (int)(v % (n + 1));
  c[1] = (int)((v / (n + 1)) % (n + 1));
  c[2] = (int)(v / ((int64_t)(n + 1) * (n + 1)));
}

// One row of the integer Galerkin parts: sorted column DOFs and the K, M, B integers.
struct RowInts {
  int m = 0;
  int32_t cols[36];
  int ik[36], im[36], ib[36];
  __device__ void add(int32_t cd, int kk, int mm, int bb) {
    // insert in column order, merging duplicates (integer sums are exact)
    int j = 0;
    while (j < m && cols[j] < cd) ++j;
    if (j < m && cols[j] == cd) {
      ik[j] += kk;
      im[j] += mm;
      ib[j] += bb;
    } else {
      for (int s = m; s > j; --s) { cols[s] = cols[s - 1]; ik[s] = ik[s - 1]; im[s] = im[s - 1]; ib[s] = ib[s - 1]; }
      cols[j] = cd; ik[j] = kk; im[j] = mm; ib[j] = bb;
      ++m;
    }
  }
};

// Row of the edge (c, d) over the tetrahedra inside the box [blo, bhi] and, with `faces`,
// the triangles on the box surface (each met once: its other tetrahedron is outside).
__device__ inline void row_ints(int n, const int* c, int d, const int* blo, const int* bhi, bool faces,
                                const int32_t* tet2dof, RowInts& R) {
  int64_t tets[6];
  int loc[6];
  const int nt = edge_tets(n, c, d, tets, loc, blo, bhi);
  for (int t = 0; t < nt; ++t) {
    const int p = (int)(tets[t] % 6);
    for (int eb = 0; eb < 6; ++eb) {
      const int32_t cd = tet2dof[tets[t] * 6 + eb];
      if (cd < 0) continue;
      int kk, mm;
      elem_int(p, loc[t], eb, kk, mm);
      R.add(cd, kk, mm, 0);
    }
    if (!faces) continue;
    const int64_t cube = tets[t] / 6;
    int V[4][3];
    V[0][0] = (int)(cube % n);
    V[0][1] = (int)((cube / n) % n);
    V[0][2] = (int)(cube / ((int64_t)n * n));
    for (int k = 0; k < 3; ++k) {
      for (int a = 0; a < 3; ++a) V[k + 1][a] = V[k][a];
      V[k + 1][a_perms[p][k]] += 1;
    }
    const int P = a_ledge[loc[t]][0], Q = a_ledge[loc[t]][1];
    for (int S = 0; S < 4; ++S) {
      if (S == P || S == Q) continue;
      for (int ax = 0; ax < 3; ++ax) {
        const int v = V[P][ax];
        if (V[Q][ax] != v || V[S][ax] != v || (v != blo[ax] && v != bhi[ax])) continue;
        // triangle {P, Q, S} on the box face normal to ax
        const int fe[3] = {loc[t], ledge_index(min(P, S), max(P, S)), ledge_index(min(Q, S), max(Q, S))};
        for (int f = 0; f < 3; ++f) {
          const int32_t cd = tet2dof[tets[t] * 6 + fe[f]];
          if (cd >= 0) R.add(cd, 0, 0, face_int(p, loc[t], fe[f], ax));
        }
      }
    }
  }
}

struct AsmArgs {
  int n;
  int64_t n_dof;
  double sK, sM, sB;
  int boundary;
  const int32_t* dof_key;
  const int32_t* tet2dof;
  int32_t* count;
  const int32_t* rowptr;
  int32_t* col;
  double* K;
  double* M;
  double* B;
};

template <bool FILL>
__global__ void k_assemble(AsmArgs a) {
  const int blo[3] = {0, 0, 0}, bhi[3] = {a.n, a.n, a.n};
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < a.n_dof;
       row += (int64_t)gridDim.x * blockDim.x) {
    int c[3], d;
    key_to_coords(a.dof_key[row], a.n, c, d);
    RowInts R;
    row_ints(a.n, c, d, blo, bhi, a.boundary != 0, a.tet2dof, R);
    if (!FILL) {
      a.count[row] = R.m;
    } else {
      const int32_t o = a.rowptr[row];
      for (int j = 0; j < R.m; ++j) {
        a.col[o + j] = R.cols[j];
        a.K[o + j] = a.sK * (double)R.ik[j];
        a.M[o + j] = a.sM * (double)R.im[j];
        if (a.B) a.B[o + j] = a.sB * (double)R.ib[j];
      }
    }
  }
}

void assemble_KM(const MeshDev& m, CsrKM& A, cudaStream_t s, bool boundary) {
  const double h = 1.0 / m.n;
  AsmArgs a{m.n, m.n_dof, 2.0 / (3.0 * h), h / 120.0, 1.0 / 24.0, boundary ? 1 : 0, m.dof_key.p, m.tet2dof.p,
            nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  DevBuf<int32_t> cnt(std::max<int64_t>(m.n_dof, 1));
  A.rows = A.cols = m.n_dof;
  A.rowptr.alloc(m.n_dof + 1);
  a.count = cnt.p;
  MX_LAUNCH(k_assemble<false><<<grid_for(m.n_dof, 128), 128, 0, s>>>(a));
  MX_CHECK_LAUNCH();
  A.nnz = exclusive_scan_i32(cnt.p, A.rowptr.p, m.n_dof, s);
  A.col.alloc(A.nnz);
  A.K.alloc(A.nnz);
  A.M.alloc(A.nnz);
  a.rowptr = A.rowptr.p;
  a.col = A.col.p;
  a.K = A.K.p;
  a.M = A.M.p;
  if (boundary) {
    A.B.alloc(A.nnz);
    a.B = A.B.p;
  } else {
    A.B.reset();
  }
  MX_LAUNCH(k_assemble<true><<<grid_for(m.n_dof, 128), 128, 0, s>>>(a));
  MX_CHECK_LAUNCH();
  MX_CUDA(cudaStreamSynchronize(s));
}

// ---- load vector --------------------------------------------------------------------
// Conical-product Gauss-Legendre rule on the reference tetrahedron, 3 points per
// direction: xi1 = u, xi2 = (1-u) v, xi3 = (1-u)(1-v) w, weight W_u W_v W_w (1-u)^2 (1-v);
// reference vertex m is path vertex m. Nodes (1 -+ sqrt(3/5))/2, 1/2 with weights
// 5/18, 4/9, 5/18 on [0, 1].
struct QuadRule {
  double xi[27][3];
  double w[27];
  double cw[27][4];   // w_q h^2 lambda_k(xi_q): weight, Jacobian 6|T| = h^3 and the 1/h of the gradients
  float2 cwd[27][4];  // cw as double-floats (hi = FP32 rounding, lo = remainder)
};

static QuadRule make_rule(double h) {
  QuadRule r;
  const double s = std::sqrt(0.6);
  const double t[3] = {0.5 * (1.0 - s), 0.5, 0.5 * (1.0 + s)};
  const double wt[3] = {5.0 / 18.0, 4.0 / 9.0, 5.0 / 18.0};
  int q = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c, ++q) {
        const double u = t[a], v = t[b], w = t[c];
        r.xi[q][0] = u;
        r.xi[q][1] = (1.0 - u) * v;
        r.xi[q][2] = (1.0 - u) * (1.0 - v) * w;
        r.w[q] = wt[a] * wt[b] * wt[c] * (1.0 - u) * (1.0 - u) * (1.0 - v);
        const double lam[4] = {1.0 - r.xi[q][0] - r.xi[q][1] - r.xi[q][2], r.xi[q][0], r.xi[q][1], r.xi[q][2]};
        for (int k = 0; k < 4; ++k) {
          r.cw[q][k] = r.w[q] * h * h * lam[k];
          const float hi = (float)r.cw[q][k];
          r.cwd[q][k] = make_float2(hi, (float)(r.cw[q][k] - (double)hi));
        }
      }
  return r;
}

struct LoadArgs {
  int n, nrhs, nbumps;
  double h, inv_w2;
  QuadRule rule;
  const double* centres;  // [nrhs][nbumps][3]
  const double2* pol;     // [nrhs][nbumps][3]
  const double* etab;     // [nrhs][nbumps][3][n][81] per-axis Gaussian factors
  float2* etab2;          // the same as double-floats (mixed form; written by k_load_table)
  const float4* pit;      // [nrhs][nbumps][6][4] p_b . g_k per path order, double-float re and im
  double2* contrib;       // [nrhs][ntet][6]
};

// The Gaussian bump is a product of one-dimensional factors, and inside cube i (per axis)
// the quadrature points' coordinates are (i + S[u]) h, u = 3q + t, with S[3q] = xi1+xi2+xi3,
// S[3q+1] = xi2+xi3, S[3q+2] = xi3 of rule point q (the path vertices add e_s0, e_s1, e_s2).
// etab[r][b][a][i][u] = exp(-((i + S[u]) h - c_{r,b,a})^2 / w^2): n * 243 exponentials per
// bump instead of one per point.
__global__ void k_load_table(LoadArgs a, double* etab) {
  const int64_t total = (int64_t)a.nrhs * a.nbumps * 3 * a.n * 81;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int u = (int)(t % 81);
    int64_t rest = t / 81;
    const int i = (int)(rest % a.n);
    rest /= a.n;
    const int ax = (int)(rest % 3);
    rest /= 3;  // = r * nbumps + b
    const int q = u / 3, tt = u % 3;
    const double s = tt == 0 ? a.rule.xi[q][0] + a.rule.xi[q][1] + a.rule.xi[q][2]
                             : (tt == 1 ? a.rule.xi[q][1] + a.rule.xi[q][2] : a.rule.xi[q][2]);
    const double d = (i + s) * a.h - a.centres[rest * 3 + ax];
    const double v = exp(-d * d * a.inv_w2);
    if (etab) etab[t] = v;
    if (a.etab2) {
      const float hi = __double2float_rn(v);
      a.etab2[t] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
  }
}

// pit[r][b][p][k] = p_b . g_k for path order p (g_0 = -e_s0, g_1 = e_s0 - e_s1, g_2 = e_s1 - e_s2,
// g_3 = e_s2; the same combinations k_load_tets forms per tetrahedron), split into double-floats
__global__ void k_load_pi(LoadArgs a, float4* pit) {
  const int total = a.nrhs * a.nbumps * 24;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int k = t % 4, p = (t / 4) % 6, rb = t / 24;
    const double2* q = a.pol + (int64_t)rb * 3;
    const double2 q0 = q[a_perms[p][0]], q1 = q[a_perms[p][1]], q2 = q[a_perms[p][2]];
    const double2 v = k == 0 ? make_double2(-q0.x, -q0.y)
                             : (k == 1 ? make_double2(q0.x - q1.x, q0.y - q1.y)
                                       : (k == 2 ? make_double2(q1.x - q2.x, q1.y - q2.y) : q2));
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    pit[t] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
  }
}

// contrib[T][a][r] = int_T F_r . w_a with the rule above (6 |T| = h^3). With w_a =
// lam_P grad lam_Q - lam_Q grad lam_P and F = sum_b p_b G_b (G_b the real Gaussian of
// bump b), the integral is sum_b (L_bP (p_b . g_Q) - L_bQ (p_b . g_P)) with the four
// weighted moments L_bk = sum_q w_q h^2 lam_k(xi_q) G_b(x_q) and g the integer gradients
// (grad lam = g / h): four FP64 FMAs per point and bump instead of a basis evaluation.
// Threads take (right-hand side, tetrahedron), tetrahedron fastest: a warp's tetrahedra lie in a
// few neighbouring cubes, so their table rows are shared or adjacent.
__global__ void k_load_tets(LoadArgs a) {
  const int64_t ntet = 6LL * a.n * a.n * a.n;
  const int64_t work = ntet * a.nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / ntet);
    const int64_t tet = t % ntet;
    const int64_t cube = tet / 6;
    const int p = (int)(tet % 6);
    const int cx = (int)(cube % a.n), cy = (int)((cube / a.n) % a.n), cz = (int)(cube / ((int64_t)a.n * a.n));
    const int s0 = a_perms[p][0], s1 = a_perms[p][1], s2 = a_perms[p][2];
    auto corner = [&](int ax) { return ax == 0 ? cx : (ax == 1 ? cy : cz); };
    // Gaussian factors from the per-axis table: the point's coordinate along axis s_t
    // (t = 0, 1, 2) is (c_{s_t} + S[3q + t]) h with S the partial sums xi1+xi2+xi3,
    // xi2+xi3, xi3 (the path starts at the cube corner c)
    const int64_t row0 = ((int64_t)s0 * a.n + corner(s0)) * 81;
    const int64_t row1 = ((int64_t)s1 * a.n + corner(s1)) * 81 + 1;
    const int64_t row2 = ((int64_t)s2 * a.n + corner(s2)) * 81 + 2;
    const double* E = a.etab + (int64_t)r * a.nbumps * 3 * a.n * 81;
    const double2* PL = a.pol + (int64_t)r * a.nbumps * 3;
    double2 acc[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) acc[e] = make_double2(0.0, 0.0);
    for (int b = 0; b < a.nbumps; ++b) {
      const double* Eb = E + (int64_t)b * 3 * a.n * 81;
      double L[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 3
      for (int q = 0; q < 27; ++q) {
        const double e = Eb[row0 + 3 * q] * Eb[row1 + 3 * q] * Eb[row2 + 3 * q];
#pragma unroll
        for (int k = 0; k < 4; ++k) L[k] = fma(a.rule.cw[q][k], e, L[k]);
      }
      // p_b . g_k with g_0 = -e_s0, g_1 = e_s0 - e_s1, g_2 = e_s1 - e_s2, g_3 = e_s2
      const double2 q0 = PL[3 * b + s0], q1 = PL[3 * b + s1], q2 = PL[3 * b + s2];
      const double2 pi[4] = {make_double2(-q0.x, -q0.y), make_double2(q0.x - q1.x, q0.y - q1.y),
                             make_double2(q1.x - q2.x, q1.y - q2.y), q2};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int P0 = e < 3 ? 0 : (e < 5 ? 1 : 2), Q0 = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
        acc[e].x += L[P0] * pi[Q0].x - L[Q0] * pi[P0].x;
        acc[e].y += L[P0] * pi[Q0].y - L[Q0] * pi[P0].y;
      }
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) a.contrib[((int64_t)r * ntet + tet) * 6 + e] = acc[e];
  }
}

// k_load_tets in double-float arithmetic on the FP32 units (mixed form): the same moments
// L_bk and edge combinations, with the Gaussian factors, weights and p_b . g_k as (hi, lo)
// FP32 pairs, products formed exactly by FMA (the lo * lo term dropped) and sums carried
// with their rounding errors. About 2^-44 relative error per moment against 2^-52 in FP64;
// the FP64 units of this GPU issue at about 1/64 of the FP32 rate.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return make_float2(p, e);
}
__global__ void k_load_tets_df(LoadArgs a) {
  const int64_t ntet = 6LL * a.n * a.n * a.n;
  const int64_t work = ntet * a.nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / ntet);
    const int64_t tet = t % ntet;
    const int64_t cube = tet / 6;
    const int p = (int)(tet % 6);
    const int cx = (int)(cube % a.n), cy = (int)((cube / a.n) % a.n), cz = (int)(cube / ((int64_t)a.n * a.n));
    const int s0 = a_perms[p][0], s1 = a_perms[p][1], s2 = a_perms[p][2];
    auto corner = [&](int ax) { return ax == 0 ? cx : (ax == 1 ? cy : cz); };
    const int64_t row0 = ((int64_t)s0 * a.n + corner(s0)) * 81;
    const int64_t row1 = ((int64_t)s1 * a.n + corner(s1)) * 81 + 1;
    const int64_t row2 = ((int64_t)s2 * a.n + corner(s2)) * 81 + 2;
    const float2* E = a.etab2 + (int64_t)r * a.nbumps * 3 * a.n * 81;
    df::Acc acc_re[6], acc_im[6];
    for (int b = 0; b < a.nbumps; ++b) {
      const float2* Eb = E + (int64_t)b * 3 * a.n * 81;
      df::Acc L[4];
#pragma unroll 3
      for (int q = 0; q < 27; ++q) {
        const float2 e = df_mul(df_mul(Eb[row0 + 3 * q], Eb[row1 + 3 * q]), Eb[row2 + 3 * q]);
#pragma unroll
        for (int k = 0; k < 4; ++k) df::add_prod2(L[k], a.rule.cwd[q][k].x, a.rule.cwd[q][k].y, e.x, e.y);
      }
      float2 Lv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) Lv[k] = df::value(L[k]);
      const float4* pi = a.pit + (((int64_t)r * a.nbumps + b) * 6 + p) * 4;
      float4 pv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) pv[k] = pi[k];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int P0 = e < 3 ? 0 : (e < 5 ? 1 : 2), Q0 = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
        // L_P (p . g_Q) - L_Q (p . g_P)
        df::add_prod2(acc_re[e], Lv[P0].x, Lv[P0].y, pv[Q0].x, pv[Q0].y);
        df::add_prod2(acc_re[e], Lv[Q0].x, Lv[Q0].y, -pv[P0].x, -pv[P0].y);
        df::add_prod2(acc_im[e], Lv[P0].x, Lv[P0].y, pv[Q0].z, pv[Q0].w);
        df::add_prod2(acc_im[e], Lv[Q0].x, Lv[Q0].y, -pv[P0].z, -pv[P0].w);
      }
    }
#pragma unroll
    for (int e = 0; e < 6; ++e)
      a.contrib[((int64_t)r * ntet + tet) * 6 + e] = make_double2(df::to_double(acc_re[e]), df::to_double(acc_im[e]));
  }
}

// f[r][i] = sum over the tetrahedra around edge i (fixed order) of contrib
__global__ void k_load_gather(int n, int64_t n_dof, int nrhs, const int32_t* dof_key,
                              const double2* contrib, double2* f) {
  const int64_t work = n_dof * nrhs;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < work;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n_dof);
    const int64_t i = t % n_dof;
    int c[3], d;
    key_to_coords(dof_key[i], n, c, d);
    int64_t tets[6];
    int loc[6];
    const int blo[3] = {0, 0, 0}, bhi[3] = {n, n, n};
    const int nt = edge_tets(n, c, d, tets, loc, blo, bhi);
    const double2* cr = contrib + (int64_t)r * 36 * n * n * n;  // 6 n^3 tetrahedra x 6 edges
    double2 s = make_double2(0, 0);
    for (int k = 0; k < nt; ++k) {
      const double2 v = cr[tets[k] * 6 + loc[k]];
      s.x += v.x;
      s.y += v.y;
    }
    f[(int64_t)r * n_dof + i] = s;
  }
}

void load_vector(const Problem& P, int nrhs, int nbumps, const double* h_centres,
                 const double* h_pol, double width, double2* f) {
  cudaStream_t s = P.stream;
  const int n = P.n;
  const int64_t ntet = 6LL * n * n * n;
  const int chunk = std::max(1, std::min(nrhs, (int)std::max<int64_t>(1, (int64_t)(512LL << 20) / (ntet * 6 * 16))));
  DevBuf<double> dc((size_t)nrhs * nbumps * 3);
  DevBuf<double2> dp((size_t)nrhs * nbumps * 3);
  MX_CUDA(cudaMemcpyAsync(dc.p, h_centres, dc.bytes(), cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemcpyAsync(dp.p, h_pol, dp.bytes(), cudaMemcpyHostToDevice, s));
  // the mixed form takes the double-float moments (k_load_tets_df), the FP64 form FP64 ones
  const bool df = P.precision == MX_MIXED;
  DevBuf<double2> contrib(ntet * 6 * chunk);
  DevBuf<double> etab(df ? 0 : (size_t)chunk * nbumps * 3 * n * 81);
  DevBuf<float2> etab2(df ? (size_t)chunk * nbumps * 3 * n * 81 : 0);
  DevBuf<float4> pit(df ? (size_t)chunk * nbumps * 24 : 0);
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int nr = std::min(chunk, nrhs - r0);
    LoadArgs a;
    a.n = n; a.nrhs = nr; a.nbumps = nbumps;
    a.h = 1.0 / n;
    a.inv_w2 = 1.0 / (width * width);
    a.rule = make_rule(1.0 / n);
    a.centres = dc.p + (int64_t)r0 * nbumps * 3;
    a.pol = dp.p + (int64_t)r0 * nbumps * 3;
    // bytes: the tetrahedron contributions written and gathered, f written; flops: 27 points x
    // (2 products + 4 FMAs) and 6 edges x 2 complex products per tetrahedron and bump
    ProfScope ps(K_LOAD, s, df ? 4 : 3, (double)ntet * 6 * 16 * 2 * nr + 16.0 * P.fine.n_dof * nr,
                 (double)ntet * nr * nbumps * (27 * 10 + 48));
    a.contrib = contrib.p;
    a.etab = df ? nullptr : etab.p;
    a.etab2 = df ? etab2.p : nullptr;
    a.pit = df ? pit.p : nullptr;
    MX_LAUNCH(k_load_table<<<grid_for((int64_t)nr * nbumps * 3 * n * 81, 256), 256, 0, s>>>(a, df ? nullptr : etab.p));
    MX_CHECK_LAUNCH();
    if (df) {
      MX_LAUNCH(k_load_pi<<<grid_for((int64_t)nr * nbumps * 24, 256), 256, 0, s>>>(a, pit.p));
      MX_LAUNCH(k_load_tets_df<<<grid_for(ntet * nr, 128), 128, 0, s>>>(a));
    } else {
      MX_LAUNCH(k_load_tets<<<grid_for(ntet * nr, 128), 128, 0, s>>>(a));
    }
    MX_CHECK_LAUNCH();
    MX_LAUNCH(k_load_gather<<<grid_for(P.fine.n_dof * nr, 256), 256, 0, s>>>(
        n, P.fine.n_dof, nr, P.fine.dof_key.p, contrib.p, f + (int64_t)r0 * P.fine.n_dof));
    MX_CHECK_LAUNCH();
  }
  MX_CUDA(cudaStreamSynchronize(s));
}

// ---- coarse restriction -------------------------------------------------------------
// (R^0)_pj = int_{e_j} w_p^H . tau ds (Eq. 3.2). The fine edge j lies in one coarse Kuhn
// simplex (meshes nested, r = n / m fine cells per coarse cell) where w_p^H is linear, so
// the midpoint rule is exact. In units of the fine half-cell the midpoint X = 2 v + D is
// an integer vector; with S = X - 2 r cube the coarse barycentrics are integer
// differences of the sorted S over 2r, and grad lam . (x_b - x_a) = (g . D) / r, so each
// entry is an integer over 2 r^2.
__device__ inline int coarse_entries(int n, int m, int32_t key, int32_t* cdof_out, int* num,
                                     const int32_t* coarse_edge_dof) {
  const int r = n / m;
  int c[3], d;
  key_to_coords(key, n, c, d);
  int X[3], cube[3], S[3];
  for (int ax = 0; ax < 3; ++ax) {
    X[ax] = 2 * c[ax] + a_dirs[d][ax];
    cube[ax] = min(X[ax] / (2 * r), m - 1);
    S[ax] = X[ax] - 2 * r * cube[ax];
  }
  // permutation sorting S in decreasing order (stable: lower axis first on ties)
  int pa[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 2 - i; ++j)
      if (S[pa[j]] < S[pa[j + 1]]) { int t = pa[j]; pa[j] = pa[j + 1]; pa[j + 1] = t; }
  // which lexicographic permutation index is this
  int p = 0;
  for (; p < 6; ++p)
    if (a_perms[p][0] == pa[0] && a_perms[p][1] == pa[1] && a_perms[p][2] == pa[2]) break;
  const int two_r = 2 * r;
  const int L[4] = {two_r - S[pa[0]], S[pa[0]] - S[pa[1]], S[pa[1]] - S[pa[2]], S[pa[2]]};
  int g[4][3];
  kuhn_grads(p, g);
  int V[4][3];
  for (int ax = 0; ax < 3; ++ax) V[0][ax] = cube[ax];
  for (int k = 0; k < 3; ++k) {
    for (int ax = 0; ax < 3; ++ax) V[k + 1][ax] = V[k][ax];
    V[k + 1][pa[k]] += 1;
  }
  int k = 0;
  const int D[3] = {a_dirs[d][0], a_dirs[d][1], a_dirs[d][2]};
  for (int e = 0; e < 6; ++e) {
    const int P0 = a_ledge[e][0], Q0 = a_ledge[e][1];
    const int numer = L[P0] * idot(g[Q0], D) - L[Q0] * idot(g[P0], D);
    if (numer == 0) continue;
    const int code = (V[Q0][0] - V[P0][0]) + 2 * (V[Q0][1] - V[P0][1]) + 4 * (V[Q0][2] - V[P0][2]);
    const int64_t v = V[P0][0] + (int64_t)(m + 1) * (V[P0][1] + (int64_t)(m + 1) * V[P0][2]);
    const int32_t cd = coarse_edge_dof[v * 7 + a_dir_of_code[code]];
    if (cd < 0) continue;
    cdof_out[k] = cd;
    num[k] = numer;
    ++k;
  }
  // sort the (<= 6) entries by coarse DOF
  for (int i = 1; i < k; ++i)
    for (int j = i; j > 0 && cdof_out[j - 1] > cdof_out[j]; --j) {
      int32_t t = cdof_out[j]; cdof_out[j] = cdof_out[j - 1]; cdof_out[j - 1] = t;
      int u = num[j]; num[j] = num[j - 1]; num[j - 1] = u;
    }
  return k;
}

template <bool FILL>
__global__ void k_r0t(int n, int m, int64_t n_dof, const int32_t* dof_key, const int32_t* cedge,
                      int32_t* count, const int32_t* rowptr, int32_t* col, double* val) {
  const double scale = 1.0 / (2.0 * (n / m) * (n / m));
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_dof;
       j += (int64_t)gridDim.x * blockDim.x) {
    int32_t cd[6];
    int num[6];
    const int k = coarse_entries(n, m, dof_key[j], cd, num, cedge);
    if (!FILL) { count[j] = k; continue; }
    const int32_t o = rowptr[j];
    for (int i = 0; i < k; ++i) {
      col[o + i] = cd[i];
      val[o + i] = scale * (double)num[i];
    }
  }
}

// R^0 rows by transposing R^0^T: one block per coarse DOF p scans the fine DOFs of the
// box of fine vertices covering the coarse cells around edge p, in increasing fine key
// order, and keeps the entries of column p (sorted by construction, no atomics).
__global__ void k_r0_rows(int n, int m, int64_t n_c, const int32_t* cdof_key, const int32_t* edge_dof,
                          const int32_t* r0t_ptr, const int32_t* r0t_col, const double* r0t_val,
                          int32_t* count, const int32_t* rowptr, int32_t* col, double* val, int fill) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t running;
  const int r = n / m;
  for (int64_t p = blockIdx.x; p < n_c; p += gridDim.x) {
    int c[3], d;
    key_to_coords(cdof_key[p], m, c, d);
    int lo[3], hi[3];
    for (int ax = 0; ax < 3; ++ax) {
      const int clo = a_dirs[d][ax] ? c[ax] : max(c[ax] - 1, 0);
      const int chi = a_dirs[d][ax] ? c[ax] + 1 : min(c[ax] + 1, m);
      lo[ax] = clo * r;
      hi[ax] = chi * r;
    }
    const int nvx = hi[0] - lo[0] + 1, nvy = hi[1] - lo[1] + 1, nvz = hi[2] - lo[2] + 1;
    const int64_t total = (int64_t)nvx * nvy * nvz * 7;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t base = 0; base < total; base += blockDim.x) {
      const int64_t t = base + threadIdx.x;
      int take = 0;
      double v = 0;
      int32_t j = -1;
      if (t < total) {
        const int dd = (int)(t % 7);
        const int64_t lv = t / 7;
        const int x = lo[0] + (int)(lv % nvx), y = lo[1] + (int)((lv / nvx) % nvy), z = lo[2] + (int)(lv / ((int64_t)nvx * nvy));
        if (x + a_dirs[dd][0] <= n && y + a_dirs[dd][1] <= n && z + a_dirs[dd][2] <= n) {
          const int64_t vid = x + (int64_t)(n + 1) * (y + (int64_t)(n + 1) * z);
          j = edge_dof[vid * 7 + dd];
          if (j >= 0) {
            for (int32_t q = r0t_ptr[j]; q < r0t_ptr[j + 1]; ++q)
              if (r0t_col[q] == (int32_t)p) { take = 1; v = r0t_val[q]; }
          }
        }
      }
      const unsigned msk = __ballot_sync(0xffffffffu, take);
      const int within = __popc(msk & ((1u << lane) - 1));
      if (lane == 0) warp_tot[warp] = __popc(msk);
      __syncthreads();
      int before = 0, all = 0;
      for (int w = 0; w < nw; ++w) {
        if (w < warp) before += warp_tot[w];
        all += warp_tot[w];
      }
      if (take && fill) {
        const int32_t o = rowptr[p] + running + before + within;
        col[o] = j;
        val[o] = v;
      }
      __syncthreads();
      if (threadIdx.x == 0) running += all;
      __syncthreads();
    }
    if (!fill && threadIdx.x == 0) count[p] = running;
    __syncthreads();
  }
}

// ---- ImpRAS local matrices ----------------------------------------------------------
struct ImpArgs {
  int n, n_sub;
  int64_t sum_local;
  double sK, sM, sB, k2, xi, c;  // A = K - (k2 + i xi) M - i c B
  const int32_t* box;            // [n_sub][6] vertex bounds
  const int64_t* offsets;
  const int32_t* lists;
  const int32_t* dof_key;
  const int32_t* tet2dof;
  const int32_t* inv_ptr;
  const int32_t* inv_pos;
  const int32_t* band;
  const int32_t* ld;
  const int64_t* moff;
  void* out;
  int32_t* bad;  // entries outside the planned band or columns outside the box (none expected)
  uint32_t* amax;  // [n_sub] largest |entry| written, as FP32 bits
};

__device__ inline uint32_t abs_bits_imp(float2 v) { return __float_as_uint(sqrtf(v.x * v.x + v.y * v.y)); }
__device__ inline uint32_t abs_bits_imp(double2 v) { return __float_as_uint((float)sqrt(v.x * v.x + v.y * v.y)); }

// One thread per (subdomain, local row): the row of the box's Galerkin matrix with the
// impedance term on the box surface, written into the band storage at the local columns.
template <typename T2>
__global__ void k_extract_imp(ImpArgs a) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < a.sum_local;
       q += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = a.n_sub - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.offsets[mid] <= q) lo = mid; else hi = mid - 1;
    }
    const int l = lo;
    const int64_t o0 = a.offsets[l], o1 = a.offsets[l + 1];
    const int i = (int)(q - o0);
    const int blo[3] = {a.box[6 * l], a.box[6 * l + 1], a.box[6 * l + 2]};
    const int bhi[3] = {a.box[6 * l + 3], a.box[6 * l + 4], a.box[6 * l + 5]};
    int c[3], d;
    key_to_coords(a.dof_key[a.lists[q]], a.n, c, d);
    RowInts R;
    row_ints(a.n, c, d, blo, bhi, true, a.tet2dof, R);
    const int bw = a.band[l], ldl = a.ld[l];
    const int64_t off = a.moff[l];
    T2* A = reinterpret_cast<T2*>(a.out);
    uint32_t amax = 0;
    for (int e = 0; e < R.m; ++e) {
      const int32_t cd = R.cols[e];
      int j = -1;
      for (int32_t t = a.inv_ptr[cd]; t < a.inv_ptr[cd + 1]; ++t) {
        const int32_t p = a.inv_pos[t];
        if (p >= o0 && p < o1) { j = (int)(p - o0); break; }
      }
      if (j < 0 || abs(i - j) > bw) {
        atomicAdd(a.bad, 1);
        continue;
      }
      const double K = a.sK * (double)R.ik[e], M = a.sM * (double)R.im[e], B = a.sB * (double)R.ib[e];
      const T2 v = conv<T2>(make_double2(K - a.k2 * M, -a.xi * M - a.c * B));
      A[bidx(off, ldl, bw, i, j)] = v;
      amax = max(amax, abs_bits_imp(v));
    }
    if (a.amax) atomicMax(a.amax + l, amax);
  }
}

void extract_imp(Problem& P) {
  cudaStream_t s = P.stream;
  const double h = 1.0 / P.n;
  DevBuf<int32_t> dbox(P.box.size()), bad(1);
  MX_CUDA(cudaMemcpyAsync(dbox.p, P.box.data(), P.box.size() * 4, cudaMemcpyHostToDevice, s));
  MX_CUDA(cudaMemsetAsync(bad.p, 0, 4, s));
  ImpArgs a{P.n, P.n_sub, P.sum_local, 2.0 / (3.0 * h), h / 120.0, 1.0 / 24.0, P.k * P.k, P.xi_prec,
            imp_coef(P, P.xi_prec), dbox.p, P.offsets.p, P.lists.p, P.fine.dof_key.p, P.fine.tet2dof.p,
            P.inv_ptr.p, P.inv_pos.p, P.band.p, P.ld.p, P.mat_off.p, P.factors.p, bad.p, P.amax.p};
  ProfScope ps(K_EXTRACT, s);
  if (P.precision == MX_MIXED)
    MX_LAUNCH(k_extract_imp<float2><<<grid_for(P.sum_local, 128), 128, 0, s>>>(a));
  else
    MX_LAUNCH(k_extract_imp<double2><<<grid_for(P.sum_local, 128), 128, 0, s>>>(a));
  MX_CHECK_LAUNCH();
  int32_t h_bad = 0;
  MX_CUDA(cudaMemcpyAsync(&h_bad, bad.p, 4, cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  MX_REQUIRE(h_bad == 0, MX_EINVAL, "impedance local matrix entry outside its subdomain band");
}

void build_coarse_restriction(Problem& P) {
  cudaStream_t s = P.stream;
  const int n = P.n, m = P.coarse_m;
  const int64_t nd = P.fine.n_dof, nc = P.coarse.n_dof;
  DevBuf<int32_t> cnt(std::max<int64_t>(nd, nc) + 1);
  P.R0T.rows = nd;
  P.R0T.cols = nc;
  P.R0T.rowptr.alloc(nd + 1);
  MX_LAUNCH(k_r0t<false><<<grid_for(nd, 256), 256, 0, s>>>(n, m, nd, P.fine.dof_key.p, P.coarse.edge_dof.p,
                                                 cnt.p, nullptr, nullptr, nullptr));
  MX_CHECK_LAUNCH();
  P.R0T.nnz = exclusive_scan_i32(cnt.p, P.R0T.rowptr.p, nd, s);
  P.R0T.col.alloc(P.R0T.nnz);
  P.R0T.val.alloc(P.R0T.nnz);
  MX_LAUNCH(k_r0t<true><<<grid_for(nd, 256), 256, 0, s>>>(n, m, nd, P.fine.dof_key.p, P.coarse.edge_dof.p,
                                                nullptr, P.R0T.rowptr.p, P.R0T.col.p, P.R0T.val.p));
  MX_CHECK_LAUNCH();
  P.R0.rows = nc;
  P.R0.cols = nd;
  P.R0.rowptr.alloc(nc + 1);
  const unsigned g = (unsigned)std::min<int64_t>(nc, 4096);
  MX_LAUNCH(k_r0_rows<<<g, 256, 0, s>>>(n, m, nc, P.coarse.dof_key.p, P.fine.edge_dof.p, P.R0T.rowptr.p,
                              P.R0T.col.p, P.R0T.val.p, cnt.p, nullptr, nullptr, nullptr, 0));
  MX_CHECK_LAUNCH();
  P.R0.nnz = exclusive_scan_i32(cnt.p, P.R0.rowptr.p, nc, s);
  MX_REQUIRE(P.R0.nnz == P.R0T.nnz, MX_EINVAL, "coarse restriction transpose mismatch");
  P.R0.col.alloc(P.R0.nnz);
  P.R0.val.alloc(P.R0.nnz);
  MX_LAUNCH(k_r0_rows<<<g, 256, 0, s>>>(n, m, nc, P.coarse.dof_key.p, P.fine.edge_dof.p, P.R0T.rowptr.p,
                              P.R0T.col.p, P.R0T.val.p, nullptr, P.R0.rowptr.p, P.R0.col.p, P.R0.val.p, 1));
  MX_CHECK_LAUNCH();
  MX_CUDA(cudaStreamSynchronize(s));
}

}  // namespace mx

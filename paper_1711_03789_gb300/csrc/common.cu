// Error state, allocation hook, launch counter, profiler and the deterministic device scan.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace mx {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

static alloc_fn g_alloc = nullptr;
static free_fn g_free = nullptr;
static void* g_ctx = nullptr;

bool allocator_hooked() { return g_alloc != nullptr; }

void set_allocator(alloc_fn a, free_fn f, void* ctx) {
  g_alloc = a;
  g_free = f;
  g_ctx = ctx;
}

void* dev_alloc(size_t bytes) {
  void* p = nullptr;
  if (g_alloc) {
    p = g_alloc(bytes, g_ctx);
    if (!p) throw Error(MX_ENOMEM, "allocator hook failed for " + std::to_string(bytes) + " bytes");
    return p;
  }
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(MX_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  if (g_free) g_free(p, g_ctx);
  else cudaFree(p);
}

// ---- launch counter and profiler ------------------------------------------------------
static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }

static const char* k_names[K_COUNT] = {
    "mesh", "subdomains", "assemble", "coarse_r0", "load_vector", "extract_minors", "lu_diag", "lu_panel",
    "lu_update", "coarse_lu", "local_solve", "coarse_restrict", "coarse_sweep", "scatter", "spmv",
    "arnoldi_dots", "arnoldi_update", "arnoldi_small", "update_x", "residual", "layout", "coarse_inverse",
    "coarse_gmres", "arnoldi_dots_c64"};
const char* kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? k_names[id] : ""; }

struct Pending {
  int id, launches;
  double bytes, flops;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<cudaEvent_t> g_pool;
static size_t g_pool_used = 0;
static std::vector<Pending> g_pending;
static double g_ms[K_COUNT], g_bytes[K_COUNT], g_flops[K_COUNT];
static int64_t g_cnt[K_COUNT];

bool prof_enabled() { return g_prof_on; }

cudaEvent_t prof_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_pool_used == g_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_pool.push_back(e);
  }
  return g_pool[g_pool_used++];
}

static thread_local int g_prof_redirect = -1;

int prof_redirect(int id) {
  const int old = g_prof_redirect;
  g_prof_redirect = id;
  return old;
}

void prof_push(int id, cudaEvent_t a, cudaEvent_t b, int launches, double bytes, double flops) {
  if (g_prof_redirect >= 0) id = g_prof_redirect;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_pending.push_back({id, launches, bytes, flops, a, b});
}

static void prof_resolve() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_pending.empty()) cudaEventSynchronize(g_pending.back().b);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) g_ms[p.id] += ms;
    g_cnt[p.id] += p.launches;
    g_bytes[p.id] += p.bytes;
    g_flops[p.id] += p.flops;
  }
  g_pending.clear();
  g_pool_used = 0;
}

void prof_reset(bool on) {
  prof_resolve();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on;
  for (int i = 0; i < K_COUNT; ++i) g_ms[i] = g_bytes[i] = g_flops[i] = 0, g_cnt[i] = 0;
}

void prof_read(double* ms, int64_t* launches, double* bytes, double* flops) {
  prof_resolve();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int i = 0; i < K_COUNT; ++i) {
    if (ms) ms[i] = g_ms[i];
    if (launches) launches[i] = g_cnt[i];
    if (bytes) bytes[i] = g_bytes[i];
    if (flops) flops[i] = g_flops[i];
  }
}

int sm_count() {
  static std::atomic<int> cached{0};  // read by the server's worker threads too
  int v = cached.load();
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
    cached.store(v);
  }
  return v;
}

// ---- exclusive scan -----------------------------------------------------------------
// Two-level scan: each block of SCAN_BLOCK threads scans SCAN_ITEMS items per thread,
// block totals are scanned recursively, then added back. Integer sums are exact, so
// the result is the same for any grid.
constexpr int SCAN_BLOCK = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T* sh, T& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  T prefix = (warp > 0 ? sh[warp - 1] : T(0)) + x - v;
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return prefix;
}

template <typename T>
__global__ void k_scan_tiles(const T* in, T* out, T* block_sums, int64_t n) {
  __shared__ T sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = (base + i < n) ? in[base + i] : T(0);
    sum += v[i];
  }
  T total;
  T pre = block_exclusive_scan<T>(sum, sh, total);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = pre;
    pre += v[i];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void k_scan_add(T* out, const T* block_pre, int64_t n) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  T add = block_pre[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + i < n) out[base + i] += add;
}

template <typename T>
static void scan_rec(const T* in, T* out, int64_t n, cudaStream_t s) {
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  DevBuf<T> sums(nb), pre(nb + 1);
  MX_LAUNCH(k_scan_tiles<T><<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, out, sums.p, n));
  MX_CHECK_LAUNCH();
  if (nb > 1) {
    scan_rec<T>(sums.p, pre.p, nb, s);
    MX_LAUNCH(k_scan_add<T><<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(out, pre.p, n));
    MX_CHECK_LAUNCH();
  }
  MX_CUDA(cudaStreamSynchronize(s));  // keep temporaries alive until done
}

template <typename T>
__global__ void k_last(const T* in, const T* out, T* dst, int64_t n) {
  dst[n] = (n > 0) ? out[n - 1] + in[n - 1] : T(0);
}

template <typename T>
static int64_t scan_impl(const T* in, T* out, int64_t n, cudaStream_t s) {
  if (n > 0) scan_rec<T>(in, out, n, s);
  MX_LAUNCH(k_last<T><<<1, 1, 0, s>>>(in, out, out, n));
  MX_CHECK_LAUNCH();
  T total = 0;
  MX_CUDA(cudaMemcpyAsync(&total, out + n, sizeof(T), cudaMemcpyDeviceToHost, s));
  MX_CUDA(cudaStreamSynchronize(s));
  return (int64_t)total;
}

int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, s);
}
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, s);
}

}  // namespace mx

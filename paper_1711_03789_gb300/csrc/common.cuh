// Shared device/host helpers of the mxas library: error handling, complex arithmetic
// on float2/double2, device buffers and a deterministic exclusive scan.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mxas.h"

namespace mx {

// ---- errors -------------------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define MX_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::mx::Error(MX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_) + \
                                      " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
  } while (0)

#define MX_CHECK_LAUNCH() MX_CUDA(cudaGetLastError())

// Every kernel launch of the library goes through MX_LAUNCH, which counts it.
void note_launch();
#define MX_LAUNCH(...)     \
  do {                     \
    __VA_ARGS__;           \
    ::mx::note_launch();   \
  } while (0)

// ---- per-kernel device timing -------------------------------------------------------
// When enabled, ProfScope brackets the launches of one step of the path with CUDA events
// on the launching stream and books their device time, launch count and algorithmic
// bytes / flops under a kernel id; mx_profile_read() resolves the events.
enum KernelId {
  K_MESH = 0, K_SUBDOMAINS, K_ASSEMBLE, K_COARSE_R0, K_LOAD, K_EXTRACT, K_LU_DIAG, K_LU_PANEL,
  K_LU_UPDATE, K_COARSE_LU, K_LOCAL_SOLVE, K_COARSE_RESTRICT, K_COARSE_SWEEP, K_SCATTER, K_SPMV,
  K_DOTS, K_ORTH_UPDATE, K_ARNOLDI_SMALL, K_UPDATE_X, K_RESIDUAL, K_LAYOUT, K_COARSE_INV, K_COARSE_GMRES, K_DOTS_C64, K_COUNT
};
const char* kernel_name(int id);
bool prof_enabled();
void prof_push(int id, cudaEvent_t a, cudaEvent_t b, int launches, double bytes, double flops);
// book every scope under `id` until restored (-1: each scope's own id); returns the previous
// setting. Used to charge a nested solve (the inner coarse GMRES) to one entry.
int prof_redirect(int id);
cudaEvent_t prof_event();

struct ProfScope {
  int id, launches;
  double bytes, flops;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(int id_, cudaStream_t s_, int launches_ = 1, double bytes_ = 0, double flops_ = 0)
      : id(id_), launches(launches_), bytes(bytes_), flops(flops_), s(s_) {
    if (prof_enabled()) {
      a = prof_event();
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event();
      cudaEventRecord(b, s);
      prof_push(id, a, b, launches, bytes, flops);
    }
  }
};

#define MX_REQUIRE(cond, code, msg)                          \
  do {                                                       \
    if (!(cond)) throw ::mx::Error((code), std::string(msg)); \
  } while (0)

// ---- complex helpers ----------------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };

__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ inline C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ inline C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ inline C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ inline C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b (4 fused multiply-adds)
template <typename C> __host__ __device__ inline void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename C> __host__ __device__ inline void cfms(C& acc, C a, C b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// 1 / a
template <typename C> __host__ __device__ inline C crcp(C a) {
  auto d = a.x * a.x + a.y * a.y;
  return mk(a.x / d, -a.y / d);
}
template <typename C> __host__ __device__ inline auto cabs2(C a) { return a.x * a.x + a.y * a.y; }

// Complex accumulation on the paired FP32 pipe (sm_100 family FFMA2): for a sum of
// products a * b keep p = sum a.x * b and q = sum a.y * b (two paired FMAs per term, no
// lane swaps); the complex sum is (p.x - q.y, p.y + q.x).
struct CAcc2 {
  float2 p, q;
};
__device__ __forceinline__ void cacc_zero(CAcc2& s) { s.p = make_float2(0.f, 0.f); s.q = s.p; }
__device__ __forceinline__ void cacc(CAcc2& s, float2 a, float2 b) {
  s.p = __ffma2_rn(make_float2(a.x, a.x), b, s.p);
  s.q = __ffma2_rn(make_float2(a.y, a.y), b, s.q);
}
__device__ __forceinline__ float2 cacc_value(const CAcc2& s) { return make_float2(s.p.x - s.q.y, s.p.y + s.q.x); }

__host__ __device__ inline float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ inline float2 to_c64(float2 a) { return a; }
__host__ __device__ inline double2 to_c128(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ inline double2 to_c128(double2 a) { return a; }
template <typename C> __host__ __device__ inline C conv(double2 a);
template <> __host__ __device__ inline double2 conv<double2>(double2 a) { return a; }
template <> __host__ __device__ inline float2 conv<float2>(double2 a) { return to_c64(a); }
template <typename C> __host__ __device__ inline C czero() { return mk(decltype(C::x)(0), decltype(C::x)(0)); }

// ---- device memory ------------------------------------------------------------------
// Allocation goes through a replaceable hook so that a host framework (for instance
// PyTorch's caching allocator) can own the memory; the default is cudaMalloc.
using alloc_fn = void* (*)(size_t bytes, void* ctx);
using free_fn = void (*)(void* p, void* ctx);
void* dev_alloc(size_t bytes);
void dev_free(void* p);

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { reset(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { reset(); }
  void alloc(size_t count) {
    reset();
    if (count) p = static_cast<T*>(dev_alloc(count * sizeof(T)));
    n = count;
  }
  // grow-only reallocation (contents are not preserved)
  void ensure(size_t count) { if (count > n) alloc(count); }
  void reset() { if (p) dev_free(p); p = nullptr; n = 0; }
  size_t bytes() const { return n * sizeof(T); }
  T* get() const { return p; }
};

// ---- launch helpers -----------------------------------------------------------------
inline unsigned grid_for(int64_t work, int block, int64_t cap = 152LL * 64) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// Deterministic exclusive scan of int32 counts (length n) into out (length n + 1,
// out[n] = total); returns the total (synchronises the stream).
int64_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);
int64_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

// number of streaming multiprocessors of the current device
int sm_count();

}  // namespace mx

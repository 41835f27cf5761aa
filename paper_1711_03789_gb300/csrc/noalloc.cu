// mx_dots_noalloc: the batched Gram-Schmidt inner products of mx_dots for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits, for instance a host
// framework that owns all device memory through its own pool and forbids side
// allocations (a side cudaMalloc would escape its accounting or fail under its fixed
// budget), or an embedding with no allocator to hand the library. mx_dots allocates its
// block partial sums per call; this variant keeps them in one fixed array in the
// library's device image instead.
//
// The scratch is the file-scope array below (4 MiB). Every GPU that loads the library
// holds it until the process exits. Its device address is looked up once per device
// with cudaGetSymbolAddress (the array's name is only a host-side stand-in in host code);
// the first call on a device performs that look-up, so make the first call before any
// stream capture. The address is kept for the life of the process, which assumes the
// device is not reset (cudaDeviceReset) in between. The call synchronises its stream
// before it returns, like mx_dots. When nvec * nrhs is above about 860 the array holds
// fewer than 2 x SM-count partial-sum blocks, so the summation order (and the last bits
// of the result) differ from mx_dots. All calls on a device share the array: calls that overlap on the GPU
// (different streams or threads without ordering) race on it. Each call rewrites every
// scratch word it later reads (partials, result, flags), so nothing has to start at zero.
#include <mutex>

#include "problem.cuh"

namespace mx {

// 4 MiB of complex128 scratch: flags (the first 16 entries, 256 B: room for 64 int32, of
// which the first nrhs <= 32 are used), then the result, then the block partials.
constexpr int64_t NOALLOC_ENTRIES = 262144;
constexpr int64_t NOALLOC_FLAG_ENTRIES = 16;
static __device__ __align__(256) double2 g_dots_scratch[NOALLOC_ENTRIES];

static std::mutex g_symbol_mu;
static double2* g_symbol_ptr[64] = {};

// Device address of g_dots_scratch for the current device (looked up once per device).
static double2* scratch_for_current_device() {
  int dev = -1;
  MX_CUDA(cudaGetDevice(&dev));
  MX_REQUIRE(dev >= 0 && dev < 64, MX_EINVAL, "device ordinal out of range for the static scratch table");
  std::lock_guard<std::mutex> lk(g_symbol_mu);
  if (!g_symbol_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_dots_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw Error(MX_ECUDA, std::string("cudaGetSymbolAddress(g_dots_scratch): ") + cudaGetErrorString(e));
    }
    g_symbol_ptr[dev] = static_cast<double2*>(p);
  }
  return g_symbol_ptr[dev];
}

static bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace mx

using namespace mx;

extern "C" MX_API int mx_dots_noalloc(const void* V, const void* w, int64_t n, int nrhs, int nvec, void* h,
                                      void* stream) {
  try {
    MX_REQUIRE(V && w && h && n >= 1 && nrhs >= 1 && nrhs <= 32 && nvec >= 1, MX_EINVAL,
               "bad mx_dots_noalloc arguments");
    const int64_t outs = (int64_t)nvec * nrhs;
    MX_REQUIRE(outs <= 16384, MX_EINVAL,
               "mx_dots_noalloc: nvec * nrhs = " + std::to_string(outs) +
                   " exceeds 16384, the most the 4 MiB static scratch holds (use mx_dots)");
    MX_REQUIRE(on_device(V) && on_device(w), MX_EINVAL, "mx_dots_noalloc: V and w must be device memory");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double2* base = scratch_for_current_device();
    int32_t* flags = reinterpret_cast<int32_t*>(base);
    double2* result = base + NOALLOC_FLAG_ENTRIES;
    double2* partials = result + ((outs + 15) / 16) * 16;
    const int64_t room = NOALLOC_ENTRIES - (partials - base);
    const int nblk = (int)std::min<int64_t>(2LL * sm_count(), room / outs);
    MX_REQUIRE(nblk >= 1, MX_EINVAL, "mx_dots_noalloc: static scratch too small");
    fill_i32(flags, nrhs, 1, s);
    batched_dots(static_cast<const double2*>(V), static_cast<const double2*>(w), n, nrhs, nvec, result, partials,
                 nblk, flags, s);
    MX_CUDA(cudaMemcpyAsync(h, result, outs * sizeof(double2), cudaMemcpyDefault, s));
    MX_CUDA(cudaStreamSynchronize(s));
    set_last_error("");
    return MX_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MX_ECUDA;
  }
}

// Allocation-free inner products for callers that cannot allocate device memory.
//
// lsweep_dots needs a handle, and a handle owns device buffers created with cudaMalloc in
// lsweep_setup.  Some callers cannot do that: code running where device allocation is not
// allowed or not wanted, such as a real-time thread that must not enter the allocator, an
// application whose memory is owned by another framework's pool, or work recorded while
// allocations are forbidden.  lsweep_dots_noalloc computes the same FP64 reductions with
// the same kernels, but its partial sums live in the fixed array below, so the call itself
// allocates nothing; the caller passes all inputs and the output.
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr int kBlocks = 304;   // reduction blocks per call (two per SM)
constexpr int kMaxK = 32;      // inner products per call (at most)

// Partial sums of one call: kMaxK x kBlocks complex128 (155,648 bytes).  The array lives in
// every GPU that loads the library until the process exits; every call shares it and
// overwrites the entries it uses, so calls that overlap on the GPU race on it.
static __device__ __align__(256) double2 g_dots_scratch[kMaxK * kBlocks];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double2* g_scratch_addr[kMaxDevices] = {};   // device address of g_dots_scratch, per device

}  // namespace

extern "C" int lsweep_dots_noalloc(const void* V, int k, int64_t n, const void* w, void* out,
                                   void* stream) {
  if (!V || !w || !out || n < 0) {
    lsw::set_global_error("lsweep_dots_noalloc: null pointer or negative length");
    return LSWEEP_EINVAL;
  }
  if (k < 1 || k > kMaxK) {
    lsw::set_global_error("lsweep_dots_noalloc: k = " + std::to_string(k) +
                          " is outside [1, 32], the capacity of its fixed scratch array");
    return LSWEEP_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    lsw::set_global_error(std::string("lsweep_dots_noalloc: no usable current device: ") +
                          cudaGetErrorString(e));
    return LSWEEP_ECUDA;
  }
  double2* scratch = nullptr;
  {
    // first call on a device, with that device current: look up the array's device address
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_dots_scratch);
      if (e != cudaSuccess || !p) {
        lsw::set_global_error(std::string("lsweep_dots_noalloc: cudaGetSymbolAddress failed: ") +
                              cudaGetErrorString(e));
        return LSWEEP_ECUDA;
      }
      g_scratch_addr[dev] = static_cast<double2*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  e = lsw::launch_dots_raw(static_cast<const double2*>(V), (long long)n, k,
                           static_cast<const double2*>(w), static_cast<double2*>(out), scratch,
                           kBlocks, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    lsw::set_global_error(std::string("lsweep_dots_noalloc: launch failed: ") +
                          cudaGetErrorString(e));
    return LSWEEP_ECUDA;
  }
  return LSWEEP_OK;
}

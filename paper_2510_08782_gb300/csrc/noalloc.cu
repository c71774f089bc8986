// Inner products without any device allocation (entry point ga_dots_noalloc of include/ga_ops.h).
//
// Some callers cannot allocate device memory: for example a program that has handed all device
// memory to its own allocator or memory pool, or a latency-critical loop that must not pay for
// cudaMalloc and the device-wide synchronisation cudaFree implies. ga_op_dots needs a context,
// and ga_setup allocates. This file gives those callers the same FP64-accurate inner products with
// their per-CTA partial sums kept in a fixed, file-scope device array instead of allocated scratch.
//
// The array is shared by every call in the process on a given device and keeps the contents of
// the last call; each call overwrites every partial it reads, so nothing has to be cleared first.
// Calls whose work overlaps on the GPU (different streams, or host threads issuing concurrently)
// race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ga.h"
#include "../../include/ga_ops.h"
#include "kernels.h"

// Room for the per-CTA partial sums of up to kNoAllocDots inner products: kNoAllocDots * kRedBlocks
// doubles = 32 * 608 * 8 bytes = 155,648 bytes, held on every device that loads the library until
// the process exits.
constexpr int kNoAllocDots = 32;
static __device__ __align__(256) double g_dot_scratch[kNoAllocDots * ga::kRedBlocks];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device. In host
// code `g_dot_scratch` names a host-side stand-in, never the device array, so it must not be passed
// to a kernel. A device reset (cudaDeviceReset, or anything else that destroys the device's primary
// context) unloads the module and frees the array, so the cached address then points at freed
// memory: the entry point must not be called on that device again in the same process.
cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ga_status ga_dots_noalloc(int prec, const void* a, const void* const* b, int count, size_t len,
                                     double* out, void* stream) {
  if (!a || !b || !out || len < 1 || (prec != GA_PREC_FP64 && prec != GA_PREC_MIXED)) {
    ga::set_global_error("ga_dots_noalloc: null pointer, empty vectors or unknown precision");
    return GA_ERR_ARG;
  }
  if (count < 1 || count > kNoAllocDots) {
    ga::set_global_error("ga_dots_noalloc: count must be between 1 and 32 (the size of the fixed scratch array)");
    return GA_ERR_ARG;
  }
  for (int i = 0; i < count; ++i)
    if (!b[i]) {
      ga::set_global_error("ga_dots_noalloc: null vector pointer");
      return GA_ERR_ARG;
    }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e == cudaSuccess) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec == GA_PREC_FP64)
      e = ga::launch_dots<double>(static_cast<const double*>(a), reinterpret_cast<const double* const*>(b), count,
                                  (long long)len, scratch, out, st);
    else
      e = ga::launch_dots<float>(static_cast<const float*>(a), reinterpret_cast<const float* const*>(b), count,
                                 (long long)len, scratch, out, st);
  }
  if (e != cudaSuccess) {
    ga::set_global_error((std::string("ga_dots_noalloc: ") + cudaGetErrorString(e)).c_str());
    return GA_ERR_CUDA;
  }
  return GA_OK;
}

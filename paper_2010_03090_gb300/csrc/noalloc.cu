// utf8_validate_host_noalloc: validation of a host buffer that allocates
// nothing.
//
// Some callers cannot allocate GPU memory at the moment they validate: a
// service whose GPU memory is fully reserved up front by a pool or by another
// framework (a cudaMalloc would fail, or fragment the reservation), code on a
// latency-critical path where cudaMalloc/cudaFree may synchronise the whole
// device, or code that must keep a fixed, known memory footprint.
// utf8_validate_host allocates a staging buffer on first use; this variant
// instead stages through a fixed array that is part of the library image,
// so it never calls cudaMalloc, cudaFree, cudaHostAlloc or any allocator.
//
// The array (result byte + halo room + kNoAllocMaxBytes of input) is a
// file-scope __device__ variable.  Under CUDA's lazy module loading (the
// default) a device gets its copy when this file's module is loaded there,
// which the first call on that device does, and keeps it until the process
// exits.  That first call (len 0 is enough) also loads the validation
// kernels, so a caller that reserves its GPU memory up front makes it on
// every device before reserving.  Its device address is looked up once per
// device with cudaGetSymbolAddress (a host-side mention of the array names a
// host stand-in, not device memory); a set-up that fails (for example out of
// memory while the module loads) is retried by the next call.  Every call
// shares the array, so calls whose work overlaps on the GPU (other threads,
// other streams) race on it; the result byte is reset to 1 at the start of
// every call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"
#include "tune.h"
#include "utf8gpu.h"

namespace utf8gpu {

int set_thread_status(int status);  // api.cu

namespace {

constexpr uint64_t kNoAllocMaxBytes = 32ull << 20;  // largest input accepted
constexpr uint64_t kNoAllocHead = 4096;              // result byte; input starts here

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocHead + kNoAllocMaxBytes];

constexpr int kMaxDevices = 64;

struct NoAllocDevice {
  std::mutex mu;
  bool ready = false;          // set-up done (only ever goes from false to true)
  uint8_t* scratch = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  LaunchCfg cfg;
};

NoAllocDevice g_na[kMaxDevices];

// Per-device set-up, with that device current: loads this module (and with it
// the array) and the validation kernels, and looks up the array's address.
// Returns false, leaving `ready` unset so that the next call tries again, if
// any step fails.
bool setup(NoAllocDevice& d, int dev) {
  std::lock_guard<std::mutex> lock(d.mu);
  if (d.ready) return true;
  uint8_t* scratch = nullptr;
  int sms = 0;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&scratch), g_noalloc_scratch);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = preload_validate_kernels();
  if (e != cudaSuccess) {
    cudaGetLastError();  // do not leave the failure to the caller's next CUDA call
    return false;
  }
  LaunchCfg cfg;
  clamp_to_occupancy(cfg);  // defaults, no tuning cache
  d.scratch = scratch;
  d.sm_count = sms;
  d.cfg = cfg;
  d.ready = true;
  return true;
}

}  // namespace

}  // namespace utf8gpu

using namespace utf8gpu;

extern "C" bool utf8_validate_host_noalloc(const uint8_t* host_data, size_t len,
                                           cudaStream_t stream) {
  if (host_data == nullptr && len > 0) return set_thread_status(UTF8_ERR_INVALID_ARG), false;
  if (len > kNoAllocMaxBytes) return set_thread_status(UTF8_ERR_BUDGET), false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return set_thread_status(UTF8_ERR_CUDA), false;
  }
  NoAllocDevice& d = g_na[dev];
  // set-up first, so that a len 0 call prepares the device
  if (!setup(d, dev)) return set_thread_status(UTF8_ERR_CUDA), false;
  if (len == 0) return set_thread_status(UTF8_OK), true;

  uint8_t* result = d.scratch;               // starts each call at 1 (valid)
  uint8_t* staged = d.scratch + kNoAllocHead;
  uint8_t flag = 0;
  cudaError_t e = cudaMemsetAsync(result, 1, 1, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(staged, host_data, len, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = launch_validate_tiles(staged, len, 0, ~uint64_t(0), result, d.cfg, d.sm_count, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, result, 1, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return set_thread_status(UTF8_ERR_CUDA), false;
  set_thread_status(UTF8_OK);
  return flag == 1;
}

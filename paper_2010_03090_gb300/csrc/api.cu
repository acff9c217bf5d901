// The C-ABI of libutf8gpu.so (declared in include/utf8gpu.h).
//
// Host-side runtime: per-device state (SM count, launch configuration, a ring
// of result bytes in pinned host memory mapped into the device, the staging
// buffer and copy stream of the host-memory path), argument checks and status
// codes.  All validation work runs in the kernels; there is no CPU path.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>

#include "internal.h"
#include "tune.h"
#include "utf8gpu.h"

namespace utf8gpu {

namespace {

thread_local int tl_status = UTF8_OK;

inline int set_status(int s) {
  tl_status = s;
  return s;
}

constexpr int kMaxDevices = 64;
constexpr uint32_t kResultSlots = 4096;
constexpr uint32_t kInfoSlots = 1024;  // utf8_error_info slots of utf8_locate_error
constexpr uint32_t kChunkCounters = 1024;  // work counters of utf8_validate_buffers_async
constexpr uint64_t kStageChunk = 64ull << 20;   // bytes per pipelined host copy
constexpr uint64_t kStageWindow = 4ull << 30;   // largest staging buffer
constexpr int kStageEvents = 64;

// UTF8GPU_STAGE_CHUNK / UTF8GPU_STAGE_WINDOW override the two sizes (bytes),
// rounded to whole tiles.
uint64_t env_size(const char* name, uint64_t fallback, uint64_t tile) {
  const char* v = getenv(name);
  uint64_t x = (v && *v) ? strtoull(v, nullptr, 10) : fallback;
  x = (x / tile) * tile;
  return x ? x : tile;
}

struct DeviceState {
  std::once_flag once;
  int init_error = cudaSuccess;
  int sm_count = 0;
  std::mutex cfg_mu;  // guards cfg: the autotuner and cache loads replace it
  LaunchCfg cfg;
  // kResultSlots result bytes of the synchronous calls, in pinned host memory
  // mapped into the device: the host sets a slot to 1, the kernels clear it
  // on an error, the host reads it after synchronising (no copies)
  uint8_t* h_results = nullptr;
  uint8_t* dm_results = nullptr;  // the device address of h_results
  std::atomic<uint32_t> next_slot{0};
  utf8_error_info* d_info = nullptr;  // kInfoSlots error locations
  // kChunkCounters device counters from which the warps of a multi-buffer
  // launch take their chunks; each launch takes the next one and zeroes it
  unsigned* d_counters = nullptr;
  std::atomic<uint32_t> next_counter{0};
  utf8_error_info* h_info = nullptr;  // pinned mirror
  std::atomic<uint32_t> next_info{0};
  // host-memory path
  std::mutex stage_mu;
  uint8_t* d_stage = nullptr;
  uint64_t stage_cap = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copied[kStageEvents] = {};
  cudaEvent_t consumed = nullptr;
};

DeviceState g_dev[kMaxDevices];

void init_device(DeviceState& d, int dev) {
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, dev);
  if (e == cudaSuccess) {
    d.sm_count = prop.multiProcessorCount;
    d.cfg = tuned_config(prop.name, prop.multiProcessorCount);
    clamp_to_occupancy(d.cfg);
    e = cudaHostAlloc(&d.h_results, kResultSlots, cudaHostAllocMapped);
  }
  if (e == cudaSuccess)
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d.dm_results), d.h_results, 0);
  if (e == cudaSuccess) e = cudaMalloc(&d.d_info, kInfoSlots * sizeof(utf8_error_info));
  if (e == cudaSuccess) e = cudaMalloc(&d.d_counters, kChunkCounters * sizeof(unsigned));
  if (e == cudaSuccess)
    e = cudaHostAlloc(&d.h_info, kInfoSlots * sizeof(utf8_error_info), cudaHostAllocDefault);
  d.init_error = e;
}

// State of the current device, or nullptr (status set) when CUDA fails.
DeviceState* device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_status(UTF8_ERR_CUDA);
    return nullptr;
  }
  DeviceState& d = g_dev[dev];
  std::call_once(d.once, init_device, std::ref(d), dev);
  if (d.init_error != cudaSuccess) {
    set_status(UTF8_ERR_CUDA);
    return nullptr;
  }
  return &d;
}

// The device's launch configuration, copied under its lock.
LaunchCfg config_of(DeviceState& d) {
  std::lock_guard<std::mutex> lock(d.cfg_mu);
  return d.cfg;
}

int cuda_status(cudaError_t e) { return set_status(e == cudaSuccess ? UTF8_OK : UTF8_ERR_CUDA); }

// UTF8GPU_CHECK_OFFSETS=1: the batch entry points check the offsets first.
bool offsets_debug_mode() {
  static const bool on = [] {
    const char* v = getenv("UTF8GPU_CHECK_OFFSETS");
    return v != nullptr && v[0] != 0 && v[0] != '0';
  }();
  return on;
}

// Runs the offsets check on `stream` and waits for it: UTF8_OK when the
// offsets are well-formed, UTF8_ERR_INVALID_ARG when not.
int check_offsets(DeviceState* d, const int64_t* offsets, int64_t count, cudaStream_t stream) {
  const uint32_t slot = d->next_slot.fetch_add(1) % kResultSlots;
  volatile uint8_t* h = d->h_results + slot;
  *h = 1;
  std::atomic_thread_fence(std::memory_order_release);
  cudaError_t e = launch_check_offsets(offsets, count, d->dm_results + slot, d->sm_count, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_status(e);
  return set_status(*h == 1 ? UTF8_OK : UTF8_ERR_INVALID_ARG);
}

}  // namespace

// Status setter for entry points defined in other files.
int set_thread_status(int status) { return set_status(status); }

bool is_device_memory(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

LaunchCfg current_config() {
  DeviceState* d = device();
  return d ? config_of(*d) : LaunchCfg();
}

void set_current_config(const LaunchCfg& cfg) {
  DeviceState* d = device();
  if (d) {
    LaunchCfg c = cfg;
    clamp_to_occupancy(c);
    std::lock_guard<std::mutex> lock(d->cfg_mu);
    d->cfg = c;
  }
}

int current_sm_count() {
  DeviceState* d = device();
  return d ? d->sm_count : 0;
}

}  // namespace utf8gpu

using namespace utf8gpu;

extern "C" {

bool utf8_validate(const uint8_t* data, size_t len, cudaStream_t stream) {
  if (len == 0) return set_status(UTF8_OK), true;
  if (data == nullptr) return set_status(UTF8_ERR_INVALID_ARG), false;
  DeviceState* d = device();
  if (!d) return false;
  if (!is_device_memory(data)) return set_status(UTF8_ERR_INVALID_ARG), false;
  const uint32_t slot = d->next_slot.fetch_add(1) % kResultSlots;
  volatile uint8_t* h = d->h_results + slot;
  *h = 1;
  std::atomic_thread_fence(std::memory_order_release);
  cudaError_t e = launch_validate_tiles(data, len, 0, ~uint64_t(0), d->dm_results + slot,
                                        config_of(*d), d->sm_count, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_status(e), false;
  set_status(UTF8_OK);
  return *h == 1;
}

int utf8_validate_async(const uint8_t* data, size_t len, uint8_t* out_valid,
                        cudaStream_t stream) {
  if (out_valid == nullptr || (data == nullptr && len > 0))
    return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(out_valid) || (len > 0 && !is_device_memory(data)))
    return set_status(UTF8_ERR_INVALID_ARG);
  if (len == 0) return cuda_status(cudaMemsetAsync(out_valid, 1, 1, stream));
  return cuda_status(launch_validate(data, len, out_valid, config_of(*d), d->sm_count, stream));
}

int utf8_validate_buffers_async(const uint8_t* const* data, const size_t* lens, int count,
                                uint8_t* out_valid, cudaStream_t stream) {
  if (count < 0 || (count > 0 && (data == nullptr || lens == nullptr || out_valid == nullptr)))
    return set_status(UTF8_ERR_INVALID_ARG);
  if (count == 0) return set_status(UTF8_OK);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(out_valid)) return set_status(UTF8_ERR_INVALID_ARG);
  for (int i = 0; i < count; ++i)
    if (lens[i] > 0 && (data[i] == nullptr || !is_device_memory(data[i])))
      return set_status(UTF8_ERR_INVALID_ARG);
  const LaunchCfg cfg = config_of(*d);
  for (int first = 0; first < count; first += kMaxBuffersPerLaunch) {
    const int n = count - first < kMaxBuffersPerLaunch ? count - first : kMaxBuffersPerLaunch;
    unsigned* next = d->d_counters + d->next_counter.fetch_add(1) % kChunkCounters;
    const cudaError_t e = launch_buffers(data + first, lens + first, n, out_valid + first, next,
                                         cfg, d->sm_count, stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return set_status(UTF8_OK);
}

int utf8_validate_fsm_async(const uint8_t* data, size_t len, uint8_t* out_valid,
                            cudaStream_t stream) {
  if (out_valid == nullptr || (data == nullptr && len > 0))
    return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(out_valid) || (len > 0 && !is_device_memory(data)))
    return set_status(UTF8_ERR_INVALID_ARG);
  cudaError_t e = cudaMemsetAsync(out_valid, 1, 1, stream);
  if (e == cudaSuccess && len > 0) e = launch_validate_fsm(data, len, out_valid, d->sm_count, stream);
  return cuda_status(e);
}

int utf8_validate_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                        uint8_t* out_valid, cudaStream_t stream) {
  if (count < 0) return set_status(UTF8_ERR_INVALID_ARG);
  if (count == 0) return set_status(UTF8_OK);
  if (data == nullptr || offsets == nullptr || out_valid == nullptr)
    return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(data) || !is_device_memory(offsets) || !is_device_memory(out_valid))
    return set_status(UTF8_ERR_INVALID_ARG);
  if (offsets_debug_mode() && check_offsets(d, offsets, count, stream) != UTF8_OK)
    return utf8_last_error();
  return cuda_status(launch_batch(data, offsets, count, out_valid, config_of(*d), d->sm_count, stream));
}

int utf8_validate_batch_desc(const utf8_batch_desc* desc, cudaStream_t stream) {
  if (desc == nullptr) return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(desc)) return set_status(UTF8_ERR_INVALID_ARG);
  return cuda_status(launch_batch_desc(desc, config_of(*d), d->sm_count, stream));
}

int utf8_check_offsets(const int64_t* offsets, int64_t count, cudaStream_t stream) {
  if (count < 0 || offsets == nullptr) return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(offsets)) return set_status(UTF8_ERR_INVALID_ARG);
  return check_offsets(d, offsets, count, stream);
}

int utf8_locate_error_async(const uint8_t* data, size_t len, utf8_error_info* out,
                            cudaStream_t stream) {
  if (out == nullptr || (data == nullptr && len > 0) ||
      (reinterpret_cast<uintptr_t>(out) & 7) != 0)
    return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(out) || (len > 0 && !is_device_memory(data)))
    return set_status(UTF8_ERR_INVALID_ARG);
  return cuda_status(launch_locate(data, len, out, config_of(*d), d->sm_count, stream));
}

int utf8_locate_error(const uint8_t* data, size_t len, utf8_error_info* out_host,
                      cudaStream_t stream) {
  if (out_host == nullptr || (data == nullptr && len > 0)) return set_status(UTF8_ERR_INVALID_ARG);
  if (len == 0) {
    out_host->position = 0;
    out_host->rule = UTF8_RULE_NONE;
    out_host->reserved = 0;
    return set_status(UTF8_OK);
  }
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(data)) return set_status(UTF8_ERR_INVALID_ARG);
  const uint32_t slot = d->next_info.fetch_add(1) % kInfoSlots;
  cudaError_t e = launch_locate(data, len, d->d_info + slot, config_of(*d), d->sm_count, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d->h_info + slot, d->d_info + slot, sizeof(utf8_error_info),
                        cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_status(e);
  *out_host = d->h_info[slot];
  return set_status(UTF8_OK);
}

int utf8_locate_errors_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                             utf8_error_info* out, cudaStream_t stream) {
  if (count < 0) return set_status(UTF8_ERR_INVALID_ARG);
  if (count == 0) return set_status(UTF8_OK);
  if (data == nullptr || offsets == nullptr || out == nullptr ||
      (reinterpret_cast<uintptr_t>(out) & 7) != 0)
    return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(data) || !is_device_memory(offsets) || !is_device_memory(out))
    return set_status(UTF8_ERR_INVALID_ARG);
  if (offsets_debug_mode() && check_offsets(d, offsets, count, stream) != UTF8_OK)
    return utf8_last_error();
  return cuda_status(launch_locate_batch(data, offsets, count, out, config_of(*d), d->sm_count, stream));
}

bool utf8_validate_host(const uint8_t* host_data, size_t len, cudaStream_t stream) {
  if (len == 0) return set_status(UTF8_OK), true;
  if (host_data == nullptr) return set_status(UTF8_ERR_INVALID_ARG), false;
  DeviceState* d = device();
  if (!d) return false;
  std::lock_guard<std::mutex> lock(d->stage_mu);
  cudaError_t e = cudaSuccess;
  const LaunchCfg cfg = config_of(*d);
  const uint64_t tb = tile_bytes(cfg);
  const uint64_t chunk = env_size("UTF8GPU_STAGE_CHUNK", kStageChunk, tb);
  const uint64_t max_window = env_size("UTF8GPU_STAGE_WINDOW", kStageWindow, chunk);
  // staging buffer: one halo tile + a window of whole chunks
  const uint64_t window = len < max_window ? ((len + tb - 1) / tb) * tb : max_window;
  const uint64_t need = tb + window;
  if (d->stage_cap < need) {
    if (d->d_stage) cudaFree(d->d_stage);
    d->d_stage = nullptr;
    d->stage_cap = 0;
    e = cudaMalloc(&d->d_stage, need);
    if (e != cudaSuccess) return cudaGetLastError(), set_status(UTF8_ERR_NOMEM), false;
    d->stage_cap = need;
  }
  if (!d->copy_stream) {
    e = cudaStreamCreateWithFlags(&d->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i < kStageEvents; ++i)
      e = cudaEventCreateWithFlags(&d->copied[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->consumed, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e), false;
  }
  const uint32_t slot = d->next_slot.fetch_add(1) % kResultSlots;
  uint8_t* result = d->dm_results + slot;
  volatile uint8_t* h = d->h_results + slot;
  *h = 1;
  std::atomic_thread_fence(std::memory_order_release);
  // Window k holds host bytes [k*window, ...) at d_stage + tb, preceded by the
  // tile of bytes before it (the halo) for k >= 1.
  uint64_t chunk_id = 0;
  for (uint64_t w0 = 0; e == cudaSuccess && w0 < len; w0 += window) {
    const uint64_t wlen = len - w0 < window ? len - w0 : window;
    const bool last_window = w0 + wlen == len;
    const uint8_t* span_data = w0 == 0 ? d->d_stage + tb : d->d_stage;
    const uint64_t span_n = w0 == 0 ? wlen : tb + wlen;
    const uint64_t first_tile = w0 == 0 ? 0 : 1;
    if (w0 > 0) {  // the previous window's kernels must be done with the buffer
      e = cudaEventRecord(d->consumed, stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(d->copy_stream, d->consumed, 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d->d_stage, host_data + w0 - tb, tb, cudaMemcpyHostToDevice,
                            d->copy_stream);
    }
    for (uint64_t c0 = 0; e == cudaSuccess && c0 < wlen; c0 += chunk) {
      const uint64_t clen = wlen - c0 < chunk ? wlen - c0 : chunk;
      const bool last_chunk = last_window && c0 + clen == wlen;
      e = cudaMemcpyAsync(d->d_stage + tb + c0, host_data + w0 + c0, clen,
                          cudaMemcpyHostToDevice, d->copy_stream);
      cudaEvent_t ev = d->copied[chunk_id++ % kStageEvents];
      if (e == cudaSuccess) e = cudaEventRecord(ev, d->copy_stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev, 0);
      // tiles of the span that end inside the copied bytes (all remaining ones,
      // padding included, after the last chunk)
      const uint64_t done = (w0 == 0 ? 0 : tb) + c0 + clen;
      const uint64_t t_begin = first_tile + (c0 / tb);
      const uint64_t t_end = last_chunk ? ~uint64_t(0) : done / tb;
      if (e == cudaSuccess)
        e = launch_validate_tiles(span_data, span_n, t_begin, t_end, result, cfg, d->sm_count,
                                  stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_status(e), false;
  set_status(UTF8_OK);
  return *h == 1;
}

int utf8_copy_validate(uint8_t* dst, const uint8_t* src, size_t len, uint8_t* out_valid,
                       cudaStream_t stream) {
  if (out_valid == nullptr || ((dst == nullptr || src == nullptr) && len > 0))
    return set_status(UTF8_ERR_INVALID_ARG);
  const uintptr_t d = reinterpret_cast<uintptr_t>(dst), s = reinterpret_cast<uintptr_t>(src);
  if (len > 0 && d < s + len && s < d + len) return set_status(UTF8_ERR_INVALID_ARG);  // overlap
  DeviceState* dev = device();
  if (!dev) return UTF8_ERR_CUDA;
  if (!is_device_memory(out_valid) || (len > 0 && (!is_device_memory(dst) || !is_device_memory(src))))
    return set_status(UTF8_ERR_INVALID_ARG);
  return cuda_status(
      launch_copy_validate(dst, src, len, out_valid, config_of(*dev), dev->sm_count, stream));
}

int utf8_classify_debug(const uint8_t* data, size_t len, uint8_t* out_special,
                        uint8_t* out_cont, cudaStream_t stream) {
  if (out_special == nullptr || out_cont == nullptr || (data == nullptr && len > 0))
    return set_status(UTF8_ERR_INVALID_ARG);
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  if (!is_device_memory(out_special) || !is_device_memory(out_cont) ||
      (len > 0 && !is_device_memory(data)))
    return set_status(UTF8_ERR_INVALID_ARG);
  return cuda_status(launch_classify_debug(data, len, out_special, out_cont, stream));
}

int utf8_last_error(void) { return tl_status; }

const char* utf8_error_string(int code) {
  switch (code) {
    case UTF8_OK: return "ok";
    case UTF8_ERR_INVALID_ARG: return "invalid argument";
    case UTF8_ERR_CUDA: return "CUDA error";
    case UTF8_ERR_TIMEOUT: return "device wait timed out";
    case UTF8_ERR_BUDGET: return "memory budget exceeded";
    case UTF8_ERR_NOMEM: return "out of memory";
    default: return "unknown status";
  }
}

int utf8_autotune(int flags) {
  DeviceState* d = device();
  if (!d) return UTF8_ERR_CUDA;
  return set_status(run_autotune(flags));
}

int utf8_tune_cache_load(const char* path) {
  if (path == nullptr) return set_status(UTF8_ERR_INVALID_ARG);
  return set_status(tune_cache_load(path));
}

int utf8_tune_cache_save(const char* path) {
  if (path == nullptr) return set_status(UTF8_ERR_INVALID_ARG);
  return set_status(tune_cache_save(path));
}

int utf8_config_json(char* buf, size_t cap) {
  DeviceState* d = device();
  if (!d) return -1;
  char tmp[256];
  const LaunchCfg cfg = config_of(*d);
  const int n = snprintf(tmp, sizeof tmp,
                         "{\"rows\": %d, \"blocks_per_sm\": %d, \"batch_rows\": %d, "
                         "\"batch_blocks_per_sm\": %d, \"sm_count\": %d, \"early_exit\": %d, "
                         "\"staged\": %d}",
                         cfg.rows, cfg.blocks_per_sm, cfg.batch_rows, cfg.batch_blocks_per_sm,
                         d->sm_count, early_exit_enabled() ? 1 : 0, cfg.staged ? 1 : 0);
  if (buf != nullptr && cap > 0) {
    strncpy(buf, tmp, cap - 1);
    buf[cap - 1] = 0;
  }
  set_status(UTF8_OK);
  return n;
}

int utf8_set_early_exit(int enable) {
  set_status(UTF8_OK);
  return set_early_exit(enable);
}

}  // extern "C"

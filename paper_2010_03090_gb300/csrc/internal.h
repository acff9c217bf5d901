// Internal declarations shared by the kernels and the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "utf8gpu.h"

namespace utf8gpu {

constexpr int kBlockThreads = 256;

// Host helpers of the C-ABI layer (api.cu).
int set_thread_status(int status);      // sets the calling thread's utf8_last_error()
bool is_device_memory(const void* p);   // device or managed memory (cudaPointerGetAttributes)

// Launch configuration (picked by the autotuner, or the defaults below).
struct LaunchCfg {
  int rows = 8;           // tile rows per warp (tile = rows * 512 bytes): 2, 4 or 8
  int blocks_per_sm = 8;  // resident CTAs per SM in the persistent grid
  int batch_rows = 8;     // tile rows for the batch kernel: 2, 4 or 8
  int batch_blocks_per_sm = 8;
  // 8-row single-buffer, multi-buffer, error-location and stream-chunk passes
  // stage their tiles through shared memory (tiles.cuh, StagedRun); set by
  // clamp_to_occupancy
  // once this device's kernels accept the shared memory, never read from a
  // tuning cache
  bool staged = false;
};

// Lets the staged kernels use their shared memory on the current device
// (validate.cu, buffers.cu); clamp_to_occupancy calls it.
cudaError_t prepare_staged_kernels();
cudaError_t prepare_buffers_staged();
cudaError_t prepare_locate_staged();
cudaError_t prepare_chunk_staged();
// Resident CTAs per SM of the staged single-buffer kernel (0 if it cannot run).
int staged_blocks_per_sm();

cudaError_t launch_validate(const uint8_t* data, uint64_t n, uint8_t* out_valid,
                            const LaunchCfg& cfg, int sm_count, cudaStream_t st);

// Checks virtual tiles [t_begin, t_end) of a buffer (used for chunked copies:
// the whole buffer is one stream, chunks arrive over time).  The result byte
// must have been set to 1 by the caller.
cudaError_t launch_validate_tiles(const uint8_t* data, uint64_t n, uint64_t t_begin,
                                  uint64_t t_end, uint8_t* out_valid, const LaunchCfg& cfg,
                                  int sm_count, cudaStream_t st);
uint64_t tile_bytes(const LaunchCfg& cfg);
// Loads every form of the single-buffer kernel (validate.cu).
cudaError_t preload_validate_kernels();

// Early exit of the single-buffer validation kernel (utf8_set_early_exit):
// process-wide, initially UTF8GPU_EARLY_EXIT (non-zero = on; off if unset).
bool early_exit_enabled();
int set_early_exit(int enable);  // returns the previous setting (0 or 1)

// Independent buffers in one launch, chunks interleaved across them and taken
// from the device counter *next (buffers.cu); sets out_valid[0 .. count) to 1
// and *next to 0 on the stream first.  count <= kMaxBuffersPerLaunch.
constexpr int kMaxBuffersPerLaunch = 64;
constexpr uint64_t kBuffersChunkBytes = 128 << 10;
cudaError_t launch_buffers(const uint8_t* const* data, const size_t* lens, int count,
                           uint8_t* out_valid, unsigned* next, const LaunchCfg& cfg,
                           int sm_count, cudaStream_t st);

// The paper's finite-state validator (Section 5) over one buffer (fsm.cu);
// the result byte must hold 1 before the launch.
cudaError_t launch_validate_fsm(const uint8_t* data, uint64_t n, uint8_t* out_valid, int sm_count,
                                cudaStream_t st);

cudaError_t launch_classify_debug(const uint8_t* data, uint64_t n, uint8_t* out_special,
                                  uint8_t* out_cont, cudaStream_t st);

// One independent buffer of a segment batch (segments.cu).
struct SegmentDesc {
  const uint8_t* data;
  uint64_t len;
};

uint64_t segment_tiles(const uint8_t* data, uint64_t len, const LaunchCfg& cfg);

// tile_prefix: device int64[count + 1], exclusive prefix of segment_tiles.
// out_valid[0 .. count) must hold 1 before the launch; the kernel clears the
// flags of invalid segments (it may be host memory mapped into the device).
cudaError_t launch_segments(const SegmentDesc* segs, const int64_t* tile_prefix, int64_t count,
                            uint64_t total_tiles, uint8_t* out_valid, const LaunchCfg& cfg,
                            int sm_count, cudaStream_t st);

// One chunk of a longer stream (stream.cu): prefix = the up to three bytes
// before it (natural order in bytes 1..3, b[-1] in byte 3) or, if prefix_dev
// is set, read from device memory (b[-3], b[-2], b[-1]); tail_out, if set,
// receives the stream's new last three bytes.  staged: 8-row tiles go through
// shared memory (LaunchCfg::staged of the device).
cudaError_t launch_chunk(const uint8_t* data, uint64_t n, uint32_t prefix,
                         const uint8_t* prefix_dev, int final_chunk, uint8_t* out_valid,
                         uint8_t* tail_out, int sm_count, bool staged, cudaStream_t st);

// Copies src to dst while validating it (copy.cu); result byte set by the call.
cudaError_t launch_copy_validate(uint8_t* dst, const uint8_t* src, uint64_t n, uint8_t* out_valid,
                                 const LaunchCfg& cfg, int sm_count, cudaStream_t st);
int copy_blocks_per_sm(int rows, int wanted);

cudaError_t launch_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                         uint8_t* out_valid, const LaunchCfg& cfg, int sm_count, cudaStream_t st);

// utf8_validate_batch with its arguments read from the device descriptor
// when the kernels run (batch.cu).
cudaError_t launch_batch_desc(const utf8_batch_desc* desc, const LaunchCfg& cfg, int sm_count,
                              cudaStream_t st);

// Clears *out_ok unless offsets[0] >= 0 and offsets[0 .. count] is
// non-decreasing (batch.cu).
cudaError_t launch_check_offsets(const int64_t* offsets, int64_t count, uint8_t* out_ok,
                                 int sm_count, cudaStream_t st);

// Error location (locate.cu): *out / out[count] are set to all ones, marked
// with the first erroneous position(s), then settled into utf8_error_info.
cudaError_t launch_locate(const uint8_t* data, uint64_t n, utf8_error_info* out,
                          const LaunchCfg& cfg, int sm_count, cudaStream_t st);
cudaError_t launch_locate_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                                utf8_error_info* out, const LaunchCfg& cfg, int sm_count,
                                cudaStream_t st);
// The batch pass of launch_locate_batch (batch.cu).
cudaError_t launch_batch_first_errors(const uint8_t* data, const int64_t* offsets, int64_t count,
                                      utf8_error_info* out, const LaunchCfg& cfg, int sm_count,
                                      cudaStream_t st);

}  // namespace utf8gpu

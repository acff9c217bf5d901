// Single-buffer validation kernel and the classification debug kernel.
//
// validate_kernel: a persistent grid (a multiple of the SM count) whose warps
// each take one contiguous run of tiles of the buffer (Section 6's loop, one
// loop per warp, the previous block carried in registers), OR their error
// words and clear the result byte if any lane saw an error.  The result byte
// is set to 1 beforehand on the same stream.  With early exit switched on
// (utf8_set_early_exit), warps also poll it and stop once another warp has
// cleared it, so an invalid buffer is rejected without reading all of it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <atomic>

#include "internal.h"
#include "tune.h"
#include "lookup.cuh"
#include "tiles.cuh"

namespace utf8gpu {

// Tiles [t_first, t_first + tiles) are split into one contiguous run per warp.
// Two CTAs per SM: the register form of the row-quad classification fits 128
// registers with a few bytes spilled (without the bound it takes 141, one CTA
// per SM); the staged form (STAGED: tiles through shared memory, the
// launch's dynamic shared memory holding each warp's ring) takes 124, with or
// without early exit (POLL).
template <int ROWS, bool POLL, bool STAGED = false>
__global__ void __launch_bounds__(kBlockThreads, 2) validate_kernel(Span s, uint64_t t_first,
                                                                uint64_t tiles,
                                                                uint8_t* out_valid) {
  const uint64_t warps = (uint64_t)gridDim.x * (kBlockThreads / kLanes);
  const uint64_t w = (uint64_t)blockIdx.x * (kBlockThreads / kLanes) + (threadIdx.x / kLanes);
  const uint64_t t0 = t_first + tiles * w / warps;
  const uint64_t t1 = t_first + tiles * (w + 1) / warps;
  uint32_t err;
  if constexpr (STAGED) {
    extern __shared__ uint4 validate_rings[];
    uint4* ring = validate_rings + (threadIdx.x / kLanes) * kStages * ROWS * kLanes;
    if constexpr (POLL) err = warp_check_tiles_staged_polling<ROWS>(s, t0, t1, ring, out_valid);
    else err = warp_check_tiles_staged<ROWS>(s, t0, t1, ring);
  } else if constexpr (POLL) {
    err = warp_check_tiles_polling<ROWS>(s, t0, t1, out_valid);
  } else {
    err = warp_check_tiles<ROWS>(s, t0, t1);
  }
  if (__any_sync(kFull, err != 0) && (threadIdx.x & (kLanes - 1)) == 0) clear_result(out_valid);
}

// One thread per 4-byte word of the virtual layout: the parts of each
// position's classification byte (see lookup.cuh), from the same lookups and
// the same error function as the validators.
__global__ void classify_debug_kernel(Span s, uint8_t* out_special, uint8_t* out_cont) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t words = s.granules * 4;
  if (k >= words) return;
  const WordLut prev = k == 0 ? ascii_lut() : lut_word(load_word(s, 4 * k - 4));
  const WordLut cur = lut_word(load_word(s, 4 * k));
  const uint32_t err = word_error(prev, cur);
  const uint32_t matched = __funnelshift_l(prev.prev_side, cur.prev_side, 8) & cur.cur_side;
  for (int j = 0; j < 4; ++j) {
    const uint64_t v = 4 * k + j;  // virtual position; output index v - off
    if (v < s.off || v >= s.off + s.n + 3) continue;
    const uint32_t is_cont = (cur.cur_side >> (8 * j + 6)) & 1u;
    // bit 6 of the error byte is is_cont XOR expected
    const uint32_t expected = ((err >> (8 * j + 6)) & 1u) ^ is_cont;
    out_special[v - s.off] = (uint8_t)((matched >> (8 * j)) & kSpecialBits);
    out_cont[v - s.off] = (uint8_t)(expected | (is_cont << 1));
  }
}

template <int ROWS>
static cudaError_t launch_rows(const Span& s, uint64_t t_begin, uint64_t t_end,
                               uint8_t* out_valid, const LaunchCfg& cfg, int sm_count,
                               cudaStream_t st) {
  const uint64_t all = span_tiles<ROWS>(s);
  if (t_end > all) t_end = all;
  if (t_begin >= t_end) return cudaSuccess;
  const uint64_t tiles = t_end - t_begin;
  const uint64_t warps_per_block = kBlockThreads / kLanes;
  uint64_t grid = (uint64_t)sm_count * (uint64_t)cfg.blocks_per_sm;
  const uint64_t need = (tiles + warps_per_block - 1) / warps_per_block;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  const bool poll = early_exit_enabled();
  if constexpr (ROWS == 8) {
    if (cfg.staged) {
      constexpr int smem = staged_smem_bytes<ROWS>(kBlockThreads);
      if (poll)
        validate_kernel<ROWS, true, true>
            <<<(unsigned)grid, kBlockThreads, smem, st>>>(s, t_begin, tiles, out_valid);
      else
        validate_kernel<ROWS, false, true>
            <<<(unsigned)grid, kBlockThreads, smem, st>>>(s, t_begin, tiles, out_valid);
      return cudaGetLastError();
    }
  }
  if (poll) {
    validate_kernel<ROWS, true><<<(unsigned)grid, kBlockThreads, 0, st>>>(s, t_begin, tiles, out_valid);
    return cudaGetLastError();
  }
  validate_kernel<ROWS, false><<<(unsigned)grid, kBlockThreads, 0, st>>>(s, t_begin, tiles, out_valid);
  return cudaGetLastError();
}

namespace {
std::atomic<int> g_early_exit{-1};  // -1: UTF8GPU_EARLY_EXIT not read yet
}  // namespace

bool early_exit_enabled() {
  int v = g_early_exit.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("UTF8GPU_EARLY_EXIT");
    int unset = -1;
    g_early_exit.compare_exchange_strong(unset, (e != nullptr && atoi(e) != 0) ? 1 : 0);
    v = g_early_exit.load(std::memory_order_relaxed);
  }
  return v == 1;
}

int set_early_exit(int enable) {
  const int before = early_exit_enabled() ? 1 : 0;
  g_early_exit.store(enable ? 1 : 0);
  return before;
}

uint64_t tile_bytes(const LaunchCfg& cfg) {
  const int rows = (cfg.rows == 2 || cfg.rows == 8) ? cfg.rows : 4;
  return (uint64_t)rows * kLanes * 16;
}

cudaError_t launch_validate_tiles(const uint8_t* data, uint64_t n, uint64_t t_begin,
                                  uint64_t t_end, uint8_t* out_valid, const LaunchCfg& cfg,
                                  int sm_count, cudaStream_t st) {
  const Span s = make_span(data, n);
  int rows = cfg.rows;
  // A whole buffer so small that its 1 KiB tiles number at most the warps of
  // the persistent grid is checked in 1 KiB tiles: larger tiles would leave
  // SMs idle.  (A range of tiles keeps the configured height, in which the
  // caller counts its tiles.)
  if (t_begin == 0 && t_end == ~uint64_t(0) && rows != 2) {
    const uint64_t grid_warps =
        (uint64_t)sm_count * (uint64_t)cfg.blocks_per_sm * (kBlockThreads / kLanes);
    if (span_tiles<2>(s) <= grid_warps) rows = 2;
  }
  switch (rows) {
    case 2: return launch_rows<2>(s, t_begin, t_end, out_valid, cfg, sm_count, st);
    case 8: return launch_rows<8>(s, t_begin, t_end, out_valid, cfg, sm_count, st);
    default: return launch_rows<4>(s, t_begin, t_end, out_valid, cfg, sm_count, st);
  }
}

cudaError_t launch_validate(const uint8_t* data, uint64_t n, uint8_t* out_valid,
                            const LaunchCfg& cfg, int sm_count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out_valid, 1, 1, st);
  if (e != cudaSuccess) return e;
  return launch_validate_tiles(data, n, 0, ~uint64_t(0), out_valid, cfg, sm_count, st);
}

cudaError_t launch_classify_debug(const uint8_t* data, uint64_t n, uint8_t* out_special,
                                  uint8_t* out_cont, cudaStream_t st) {
  const Span s = make_span(data, n);
  const uint64_t words = s.granules * 4;
  const unsigned block = 256;
  const uint64_t grid = (words + block - 1) / block;
  classify_debug_kernel<<<(unsigned)grid, block, 0, st>>>(s, out_special, out_cont);
  return cudaGetLastError();
}

}  // namespace utf8gpu

namespace utf8gpu {

// Resident CTAs per SM that both forms of the kernel (with and without
// early exit) reach.
template <int ROWS>
static int validate_fit() {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, validate_kernel<ROWS, false>,
                                                    kBlockThreads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, validate_kernel<ROWS, true>,
                                                    kBlockThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int n = a < b ? a : b;
  return n > 0 ? n : 1;
}

// Loads every form of validate_kernel that launch_validate_tiles can launch
// (under lazy module loading a kernel is otherwise loaded at its first
// launch, which may then need device memory).
cudaError_t preload_validate_kernels() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, validate_kernel<2, false>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, validate_kernel<2, true>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, validate_kernel<4, false>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, validate_kernel<4, true>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, validate_kernel<8, false>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, validate_kernel<8, true>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, validate_kernel<8, false, true>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, validate_kernel<8, true, true>);
  return e;
}

cudaError_t prepare_staged_kernels() {
  const int smem = staged_smem_bytes<8>(kBlockThreads);
  cudaError_t e = cudaSuccess;
  for (const void* f : {reinterpret_cast<const void*>(validate_kernel<8, false, true>),
                        reinterpret_cast<const void*>(validate_kernel<8, true, true>)}) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
  }
  if (e == cudaSuccess) e = prepare_buffers_staged();
  if (e == cudaSuccess) e = prepare_locate_staged();
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

// (the smaller of the forms with and without early exit)
int staged_blocks_per_sm() {
  const int smem = staged_smem_bytes<8>(kBlockThreads);
  int n = 0, m = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, validate_kernel<8, false, true>,
                                                    kBlockThreads, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, validate_kernel<8, true, true>,
                                                    kBlockThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n < m ? n : m;
}

int validate_blocks_per_sm(int rows) {
  switch (rows) {
    case 2: return validate_fit<2>();
    case 8: return validate_fit<8>();
    default: return validate_fit<4>();
  }
}

}  // namespace utf8gpu

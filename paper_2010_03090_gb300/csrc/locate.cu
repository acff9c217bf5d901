// Error location for one buffer and for batches (see locate.cuh).
//
// locate_kernel streams the buffer exactly like validate_kernel (same tiles,
// persistent grid, one contiguous run of tiles per warp, next tile prefetched)
// and, on the first tile of its run that holds an error, takes the warp's
// smallest erroneous position into an atomic minimum and stops: its later
// tiles can only hold larger positions.  A one-thread kernel then settles the
// minimum into the location.  For batches the batch pass (batch.cu) marks each
// string's first erroneous position and one thread per string settles it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "locate.cuh"
#include "lookup.cuh"
#include "tiles.cuh"

namespace utf8gpu {

// Two CTAs per SM: with row quads and register loads the kernel fits 128
// registers with a few bytes spilled (160 without the bound, one CTA per SM
// and 2.4% slower than row pairs; with the bound 3% faster than row pairs).
// STAGED: the tiles come through the warp's ring in the launch's dynamic
// shared memory (StagedRun, tiles.cuh), two tiles ahead.
template <int ROWS, bool STAGED = false>
__global__ void __launch_bounds__(kBlockThreads, 2)
    locate_kernel(Span s, uint64_t tiles, utf8_error_info* out) {
  constexpr uint64_t tb = TileGeom<ROWS>::kBytes;
  const int lane = threadIdx.x & (kLanes - 1);
  const uint64_t warps = (uint64_t)gridDim.x * (kBlockThreads / kLanes);
  const uint64_t w = (uint64_t)blockIdx.x * (kBlockThreads / kLanes) + (threadIdx.x / kLanes);
  const uint64_t t0 = tiles * w / warps;
  const uint64_t t1 = tiles * (w + 1) / warps;
  if (t0 >= t1) return;
  const uint32_t merge_sel = carry_merge_selector<kQuadRows<ROWS>>(lane);
  Carry carry = ascii_carry();
  if (t0 > 0) carry = halo_carry<kQuadRows<ROWS>>(load_word(s, t0 * tb - 4));
  const RunTiles run = run_tiles<ROWS>(s, t0, t1);
  const uint8_t* lane_ptr = s.abase + t0 * tb + lane * 16;
  // Every kPollBytes the warp looks at the smallest position marked so far
  // (loaded kPollBytes earlier, so the load's latency stays hidden): once it
  // lies before the warp's next tile, no error the warp could still find is
  // the first, and the warp stops.
  constexpr uint32_t poll_tiles = kPollBytes / (uint32_t)tb;
  static_assert(poll_tiles >= 1, "a poll falls after whole tiles");
  const bool poll = poll_tiles < run.cnt;
  uint64_t best = poll ? load_position(out) : ~uint64_t(0);
  uint4 next[STAGED ? 1 : ROWS];
  extern __shared__ uint4 locate_rings[];
  StagedRun<ROWS> ring(s, t0, t1, locate_rings + (threadIdx.x / kLanes) * kStages * ROWS * kLanes,
                       lane);
  if constexpr (STAGED) ring.start();
  else load_run_tile<ROWS>(s, run, t0, 0, lane, lane_ptr, next);
  uint32_t tiles_to_look = poll_tiles;
  for (uint32_t k = 0; k < run.cnt; ++k, lane_ptr += tb) {
    uint4 d[ROWS];
    if constexpr (STAGED) {
      ring.next(k, d);
    } else {
#pragma unroll
      for (int r = 0; r < ROWS; ++r) d[r] = next[r];
      if (k + 1 < run.cnt) load_run_tile<ROWS>(s, run, t0, k + 1, lane, lane_ptr + tb, next);
    }
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS>(d, carry, lane, merge_sel, e);
    uint32_t any = 0;
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) any |= e[p][m];
    if (__any_sync(kFull, any != 0)) {
      const uint32_t first = __reduce_min_sync(kFull, lane_first_error<ROWS>(e, lane));
      // virtual positions before s.off are zeros after zeros: never erroneous
      if (lane == 0) mark_first_error(out, (t0 + k) * tb + first - s.off);
      if constexpr (STAGED) ring.finish();
      return;
    }
    if (poll && --tiles_to_look == 0) {  // (t0 + k + 1) * tb > s.off here
      tiles_to_look = poll_tiles;
      if (__any_sync(kFull, best < (t0 + k + 1) * tb - s.off)) {
        if constexpr (STAGED) ring.finish();
        return;
      }
      best = load_position(out);
    }
  }
  if constexpr (STAGED) ring.finish();
}

__global__ void settle_kernel(const uint8_t* data, uint64_t n, utf8_error_info* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) settle_location(data, n, out->position, out);
}

__global__ void settle_batch_kernel(const uint8_t* __restrict__ data,
                                    const int64_t* __restrict__ offsets, int64_t count,
                                    utf8_error_info* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const int64_t o = offsets[i];
    settle_location(data + o, (uint64_t)(offsets[i + 1] - o), out[i].position, &out[i]);
  }
}

template <int ROWS, bool STAGED>
static int locate_occupancy() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, locate_kernel<ROWS, STAGED>, kBlockThreads,
          STAGED ? staged_smem_bytes<ROWS>(kBlockThreads) : 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

template <int ROWS, bool STAGED = false>
static cudaError_t launch_locate_rows(const Span& s, utf8_error_info* out, int blocks_per_sm,
                                      int sm_count, cudaStream_t st) {
  const uint64_t tiles = span_tiles<ROWS>(s);
  const int fit = locate_occupancy<ROWS, STAGED>();
  const int bps = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : fit;
  const uint64_t warps_per_block = kBlockThreads / kLanes;
  uint64_t grid = (uint64_t)sm_count * (uint64_t)bps;
  const uint64_t need = (tiles + warps_per_block - 1) / warps_per_block;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  locate_kernel<ROWS, STAGED>
      <<<(unsigned)grid, kBlockThreads, STAGED ? staged_smem_bytes<ROWS>(kBlockThreads) : 0, st>>>(
          s, tiles, out);
  return cudaGetLastError();
}

cudaError_t prepare_locate_staged() {
  const int smem = staged_smem_bytes<8>(kBlockThreads);
  cudaError_t e = cudaFuncSetAttribute(locate_kernel<8, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(locate_kernel<8, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t launch_locate(const uint8_t* data, uint64_t n, utf8_error_info* out,
                          const LaunchCfg& cfg, int sm_count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0xFF, sizeof(utf8_error_info), st);
  if (e == cudaSuccess && n > 0) {
    const Span s = make_span(data, n);
    switch (cfg.rows) {
      case 2: e = launch_locate_rows<2>(s, out, cfg.blocks_per_sm, sm_count, st); break;
      case 4: e = launch_locate_rows<4>(s, out, cfg.blocks_per_sm, sm_count, st); break;
      default:
        e = cfg.staged ? launch_locate_rows<8, true>(s, out, cfg.blocks_per_sm, sm_count, st)
                       : launch_locate_rows<8>(s, out, cfg.blocks_per_sm, sm_count, st);
        break;
    }
  }
  if (e != cudaSuccess) return e;
  settle_kernel<<<1, 32, 0, st>>>(data, n, out);
  return cudaGetLastError();
}

cudaError_t launch_locate_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                                utf8_error_info* out, const LaunchCfg& cfg, int sm_count,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0xFF, (size_t)count * sizeof(utf8_error_info), st);
  if (e == cudaSuccess) e = launch_batch_first_errors(data, offsets, count, out, cfg, sm_count, st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (count + 255) / 256;
  const int64_t cap = (int64_t)sm_count * 8;
  settle_batch_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, st>>>(data, offsets,
                                                                              count, out);
  return cudaGetLastError();
}

}  // namespace utf8gpu

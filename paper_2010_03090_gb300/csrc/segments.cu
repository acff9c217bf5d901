// Many independent buffers in one launch (the serving path's batches).
//
// Segment i is the buffer segs[i].data[0 .. segs[i].len), checked on its own
// exactly as utf8_validate checks one buffer.  tile_prefix[i] is the number
// of tiles of segments 0..i-1 (tiles of each segment's own 16-byte aligned
// layout, padding included), so the batch is one range of tiles that the
// persistent grid splits evenly across warps: a warp may cover the end of
// one segment and the start of the next, and a large segment is shared by
// many warps, each starting from the 4 bytes before its first tile.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "lookup.cuh"
#include "tiles.cuh"
#include "tune.h"

namespace utf8gpu {

template <int ROWS>
__global__ void __launch_bounds__(kBlockThreads)
    segments_kernel(const SegmentDesc* __restrict__ segs, const int64_t* __restrict__ tile_prefix,
                    int64_t count, uint8_t* __restrict__ out_valid) {
  const int lane = threadIdx.x & (kLanes - 1);
  const uint64_t warps = (uint64_t)gridDim.x * (kBlockThreads / kLanes);
  const uint64_t w = (uint64_t)blockIdx.x * (kBlockThreads / kLanes) + (threadIdx.x / kLanes);
  const uint64_t total = (uint64_t)tile_prefix[count];
  const uint64_t t0 = total * w / warps;
  const uint64_t t1 = total * (w + 1) / warps;
  if (t0 >= t1) return;
  // last segment with tile_prefix[i] <= t0 (binary search, uniform per warp)
  int64_t lo = 0, hi = count;  // tile_prefix[lo] <= t0 < tile_prefix[hi]
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if ((uint64_t)tile_prefix[mid] <= t0) lo = mid; else hi = mid;
  }
  for (int64_t i = lo; i < count && (uint64_t)tile_prefix[i] < t1; ++i) {
    const uint64_t base = (uint64_t)tile_prefix[i];
    const uint64_t end = (uint64_t)tile_prefix[i + 1];
    const uint64_t a = (t0 > base ? t0 : base) - base;
    const uint64_t b = (t1 < end ? t1 : end) - base;
    if (a >= b) continue;
    const Span s = make_span(segs[i].data, segs[i].len);
    const uint32_t err = warp_check_tiles<ROWS, false>(s, a, b);
    if (__any_sync(kFull, err != 0) && lane == 0) clear_result(out_valid + i);
  }
}

uint64_t segment_tiles(const uint8_t* data, uint64_t len, const LaunchCfg& cfg) {
  const Span s = make_span(data, len);
  switch (cfg.rows) {
    case 2: return span_tiles<2>(s);
    case 8: return span_tiles<8>(s);
    default: return span_tiles<4>(s);
  }
}

cudaError_t launch_segments(const SegmentDesc* segs, const int64_t* tile_prefix, int64_t count,
                            uint64_t total_tiles, uint8_t* out_valid, const LaunchCfg& cfg,
                            int sm_count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const uint64_t warps_per_block = kBlockThreads / kLanes;
  uint64_t grid = (uint64_t)sm_count * (uint64_t)cfg.blocks_per_sm;
  const uint64_t need = (total_tiles + warps_per_block - 1) / warps_per_block;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  switch (cfg.rows) {
    case 2:
      segments_kernel<2><<<(unsigned)grid, kBlockThreads, 0, st>>>(segs, tile_prefix, count, out_valid);
      break;
    case 8:
      segments_kernel<8><<<(unsigned)grid, kBlockThreads, 0, st>>>(segs, tile_prefix, count, out_valid);
      break;
    default:
      segments_kernel<4><<<(unsigned)grid, kBlockThreads, 0, st>>>(segs, tile_prefix, count, out_valid);
  }
  return cudaGetLastError();
}

}  // namespace utf8gpu

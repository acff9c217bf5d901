// Many independent buffers validated in one launch (utf8_validate_buffers_async).
//
// Each buffer is checked exactly as utf8_validate would check it (Section 6,
// its own zero padding before and after), but the buffers share one
// persistent grid: the work is cut into chunks of consecutive tiles, the
// chunks of all buffers are interleaved in proportion to the buffers' sizes,
// and warps take chunks one at a time from a counter.  So at any moment the
// warps work on every buffer at once: a buffer whose tiles are all ASCII is
// bound by HBM bandwidth (the tile early-out leaves the ALU idle), a buffer
// of non-ASCII text by the integer ALU pipe (the classification), and the
// two kinds run side by side instead of one after the other.
//
// Interleaved order.  Buffers are sorted by chunk count, largest first.
// Round r holds chunk r of every buffer that has more than r chunks, so the
// rounds fall into at most `count` segments with a fixed set of active
// buffers; chunk c of the order is found from the segment that holds it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "tiles.cuh"

namespace utf8gpu {
namespace {

struct BuffersArgs {
  Span s[kMaxBuffersPerLaunch];
  uint8_t order[kMaxBuffersPerLaunch];      // buffer indices, most chunks first
  uint32_t seg_round[kMaxBuffersPerLaunch];  // first round of segment i
  uint32_t seg_chunk[kMaxBuffersPerLaunch + 1];  // first chunk of segment i (last: total)
  uint8_t seg_active[kMaxBuffersPerLaunch];  // buffers active in segment i: order[0 .. n)
  int segments;
  uint32_t chunk_tiles;
};

// STAGED: tiles through shared memory (the launch's dynamic shared memory
// holds each warp's ring, see warp_check_tiles_staged).
template <int ROWS, bool STAGED>
__global__ void __launch_bounds__(kBlockThreads, 2) buffers_kernel(BuffersArgs a, unsigned* next,
                                                               uint8_t* out_valid) {
  const int lane = threadIdx.x & (kLanes - 1);
  const uint32_t total = a.seg_chunk[a.segments];
  uint32_t c = 0;
  if (lane == 0) c = atomicAdd(next, 1u);
  c = __shfl_sync(kFull, c, 0);
  while (c < total) {
    // the next chunk is asked for now, its number used after this one
    uint32_t c_next = 0;
    if (lane == 0) c_next = atomicAdd(next, 1u);
    int i = 0;
    while (i + 1 < a.segments && a.seg_chunk[i + 1] <= c) ++i;
    const uint32_t in_seg = c - a.seg_chunk[i];
    const uint32_t n = a.seg_active[i];
    const int b = a.order[in_seg % n];
    const uint64_t round = (uint64_t)a.seg_round[i] + in_seg / n;
    const uint64_t all = span_tiles<ROWS>(a.s[b]);
    const uint64_t t0 = round * a.chunk_tiles;
    const uint64_t t1 = t0 + a.chunk_tiles < all ? t0 + a.chunk_tiles : all;
    uint32_t err;
    if constexpr (STAGED) {
      extern __shared__ uint4 buffers_rings[];
      err = warp_check_tiles_staged<ROWS>(
          a.s[b], t0, t1, buffers_rings + (threadIdx.x / kLanes) * kStages * ROWS * kLanes);
    } else {
      err = warp_check_tiles<ROWS>(a.s[b], t0, t1);
    }
    if (__any_sync(kFull, err != 0) && lane == 0) clear_result(out_valid + b);
    c = __shfl_sync(kFull, c_next, 0);
  }
}

template <int ROWS>
cudaError_t launch_rows(const BuffersArgs& a, unsigned* next, uint8_t* out_valid, int blocks,
                        bool staged, cudaStream_t st) {
  if constexpr (ROWS == 8) {
    if (staged) {
      buffers_kernel<ROWS, true>
          <<<(unsigned)blocks, kBlockThreads, staged_smem_bytes<ROWS>(kBlockThreads), st>>>(
              a, next, out_valid);
      return cudaGetLastError();
    }
  }
  buffers_kernel<ROWS, false><<<(unsigned)blocks, kBlockThreads, 0, st>>>(a, next, out_valid);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_buffers(const uint8_t* const* data, const size_t* lens, int count,
                           uint8_t* out_valid, unsigned* next, const LaunchCfg& cfg,
                           int sm_count, cudaStream_t st) {
  const int rows = (cfg.rows == 2 || cfg.rows == 8) ? cfg.rows : 4;
  BuffersArgs a{};
  a.chunk_tiles = (uint32_t)(kBuffersChunkBytes / tile_bytes(cfg));
  uint32_t chunks[kMaxBuffersPerLaunch];
  uint64_t sum = 0;
  for (int i = 0; i < count; ++i) {
    a.s[i] = make_span(data[i], lens[i]);
    const uint64_t tiles = rows == 2 ? span_tiles<2>(a.s[i])
                           : rows == 8 ? span_tiles<8>(a.s[i]) : span_tiles<4>(a.s[i]);
    const uint64_t ch = (tiles + a.chunk_tiles - 1) / a.chunk_tiles;
    if (ch > 0xFFFFFFFFull) return cudaErrorInvalidValue;
    chunks[i] = (uint32_t)ch;
    sum += ch;
    a.order[i] = (uint8_t)i;
  }
  if (sum > 0xFFFF0000ull) return cudaErrorInvalidValue;  // chunk numbers fit 32 bits
  std::stable_sort(a.order, a.order + count,
                   [&](uint8_t x, uint8_t y) { return chunks[x] > chunks[y]; });
  // segments: rounds [chunks of order[k+1], chunks of order[k]) have k + 1 buffers
  uint32_t round = 0, chunk = 0;
  int seg = 0;
  for (int k = count - 1; k >= 0; --k) {
    // buffers order[0 .. k] are active until round chunks[order[k]]
    const uint32_t end = chunks[a.order[k]];
    if (end <= round) continue;
    a.seg_round[seg] = round;
    a.seg_chunk[seg] = chunk;
    a.seg_active[seg] = (uint8_t)(k + 1);
    chunk += (end - round) * (uint32_t)(k + 1);
    round = end;
    ++seg;
  }
  a.segments = seg;
  a.seg_chunk[seg] = chunk;
  cudaError_t e = cudaMemsetAsync(out_valid, 1, (size_t)count, st);
  if (e != cudaSuccess || chunk == 0) return e;
  e = cudaMemsetAsync(next, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int blocks = sm_count * cfg.blocks_per_sm;
  switch (rows) {
    case 2: return launch_rows<2>(a, next, out_valid, blocks, false, st);
    case 8: return launch_rows<8>(a, next, out_valid, blocks, cfg.staged, st);
    default: return launch_rows<4>(a, next, out_valid, blocks, false, st);
  }
}

cudaError_t prepare_buffers_staged() {
  const int smem = staged_smem_bytes<8>(kBlockThreads);
  cudaError_t e = cudaFuncSetAttribute(buffers_kernel<8, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(buffers_kernel<8, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

}  // namespace utf8gpu

// Batched validation: one flag per string, all strings in one launch.
//
// The strings of a batch lie back to back in one buffer (string i is
// data[offsets[i] .. offsets[i+1])).  Instead of scheduling strings, the
// kernel streams the whole region [offsets[0], offsets[count]) exactly like
// a single buffer (same tiles, same warp routine, same persistent grid), so
// every warp gets the same number of bytes whatever the length mix, all lanes
// stay busy on short strings, and long strings are split across warps with
// the 3-byte halo stitched through the carried previous word.
//
// Streaming the concatenation checks every position with the previous bytes
// of the concatenation.  That is exact for every position at least three
// bytes after a string's start (its window lies inside the string).  The
// positions near string boundaries are checked separately and exactly, one
// lane per boundary, from the string's own bytes with the virtual zeros the
// paper puts before and after a stream (Section 6, Section 6.3):
//   head check of string j: positions o_j .. o_j+3, previous bytes zero,
//                           bytes past the string's end zero;
//   tail check of string j: positions e_j .. e_j+3 (all virtual zeros),
//                           previous bytes the string's last bytes.
// A streamed error at position p is charged to the string holding p, unless
// p lies in that string's first three bytes (the head check decides those).
// Boundary o_j is handled by the warp whose tile holds its position, so each
// is handled once; flags only ever go from 1 (set before the launch) to 0.
// With LOCATE the same checks lower each string's first erroneous position
// (an atomic minimum, string-relative) instead of clearing its flag.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tune.h"
#include "locate.cuh"
#include "lookup.cuh"
#include "search.cuh"
#include "tiles.cuh"

namespace utf8gpu {

// Bytes [x, x + 4) of `data` (absolute offsets), zero outside [lo, hi).
__device__ __forceinline__ uint32_t gather4(const uint8_t* data, int64_t x, int64_t lo,
                                            int64_t hi) {
  uint32_t w = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t y = x + k;
    if (y >= lo && y < hi) w |= (uint32_t)__ldg(data + y) << (8 * k);
  }
  return w;
}

// First j in [lo, hi) with offsets[j] >= target (hi if none); whole warp.
__device__ int64_t warp_lower_bound(const int64_t* offsets, int64_t lo, int64_t hi,
                                    int64_t target) {
  const int lane = threadIdx.x & (kLanes - 1);
  while (hi - lo > kLanes) {
    const int64_t step = lb_step(lo, hi);
    const int64_t j = lo + lane * step;
    const bool ge = j < hi ? offsets[j] >= target : true;
    const LbRange r = lb_narrow(lo, hi, step, __ballot_sync(kFull, ge));
    lo = r.lo;
    hi = r.hi;
  }
  const int64_t j = lo + lane;
  const bool ge = j < hi ? offsets[j] >= target : true;
  return lb_final(lo, hi, __ballot_sync(kFull, ge));
}

// An error at `rel` bytes into string j: its flag is cleared, or (LOCATE) its
// first erroneous position is lowered to rel (see locate.cuh).
template <bool LOCATE>
__device__ __forceinline__ void charge(uint8_t* out_valid, utf8_error_info* out_err, int64_t j,
                                       int64_t rel) {
  if constexpr (LOCATE) {
    mark_first_error(&out_err[j], (uint64_t)rel);
  } else {
    out_valid[j] = 0;
  }
}

template <int ROWS, bool LOCATE>
__global__ void __launch_bounds__(kBlockThreads)
    batch_kernel(const uint8_t* __restrict__ data, const int64_t* __restrict__ offsets,
                 int64_t count, uint8_t* __restrict__ out_valid, utf8_error_info* out_err) {
  constexpr uint64_t kTileBytes = (uint64_t)kLanes * ROWS * 16;
  // The region [offsets[0], offsets[count]) is read on the device, so the
  // launch needs nothing from the host but the pointers (graph capturable).
  const int64_t o_first = offsets[0];
  const int64_t o_last = offsets[count];
  const Span region = make_span(data + o_first, o_last > o_first ? (uint64_t)(o_last - o_first) : 0);
  const uint64_t tiles = span_tiles<ROWS>(region);
  const int lane = threadIdx.x & (kLanes - 1);
  const uint64_t warps = (uint64_t)gridDim.x * (kBlockThreads / kLanes);
  const uint64_t w = (uint64_t)blockIdx.x * (kBlockThreads / kLanes) + (threadIdx.x / kLanes);
  const uint64_t t0 = tiles * w / warps;
  const uint64_t t1 = tiles * (w + 1) / warps;
  if (t0 >= t1) return;

  // absolute offset of virtual position 0 of the region
  const int64_t vbase = o_first - (int64_t)region.off;
  const int64_t range_lo = vbase + (int64_t)(t0 * kTileBytes);
  const int64_t range_hi = vbase + (int64_t)(t1 * kTileBytes);
  // boundaries of this warp: offsets[j] in [range_lo, range_hi), j in [b0, b1)
  const int64_t b0 = warp_lower_bound(offsets, 0, count + 1, range_lo);
  const int64_t b1 = warp_lower_bound(offsets, b0, count + 1, range_hi);
  // strings that can hold a position of this warp: b0 - 1 .. b1 - 1
  const int64_t own_lo = b0 > 0 ? b0 - 1 : 0;
  const int64_t own_hi = b1 < count ? b1 : count;

  const uint32_t merge_sel = carry_merge_selector(lane);
  Carry carry = ascii_carry();
  if (t0 > 0) carry = halo_carry(load_word(region, t0 * kTileBytes - 4));
  uint64_t in0, in1;
  interior_tiles<ROWS>(region, in0, in1);
  const uint8_t* lane_ptr = region.abase + t0 * kTileBytes + lane * 16;
  int64_t next_group = b0;  // first boundary not yet checked
  int64_t group_last = (next_group + kLanes < b1 ? next_group + kLanes : b1) - 1;
  int64_t group_last_off = next_group < b1 ? offsets[group_last] : 0;
  uint4 next[ROWS];  // the next tile's loads, issued one tile ahead
  load_tile<ROWS>(region, t0, in0, in1, lane, lane_ptr, next);

  for (uint64_t t = t0; t < t1; ++t, lane_ptr += kTileBytes) {
    const int64_t tile_lo = vbase + (int64_t)(t * kTileBytes);
    const int64_t tile_hi = tile_lo + (int64_t)kTileBytes;

    // ---- stream the tile (plain `lookup` over the concatenation) ----------
    uint4 d[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) d[r] = next[r];
    if (t + 1 < t1) load_tile<ROWS>(region, t + 1, in0, in1, lane, lane_ptr + kTileBytes, next);
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS>(d, carry, lane, merge_sel, e);
    uint32_t any_err = 0;
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) any_err |= e[p][m];

    // ---- charge streamed errors to strings (only where errors exist) -----
    if (__any_sync(kFull, any_err != 0)) {
#pragma unroll
      for (int pr = 0; pr < ROWS / 2; ++pr) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          uint32_t bits = e[pr][m];
          while (bits != 0) {
            const int byte = (__ffs(bits) - 1) >> 3;
            bits &= ~(0xFFu << (8 * byte));
            const int64_t p = tile_lo + (int64_t)interleaved_position<ROWS>(pr, m, byte, lane);
            const int64_t own = last_at_most(offsets, own_lo, own_hi + 1, p);
            if (own >= 0 && own < count && p - offsets[own] >= 3 && p < offsets[own + 1])
              charge<LOCATE>(out_valid, out_err, own, p - offsets[own]);
          }
        }
      }
    }

    // ---- boundaries: exact head and tail checks, 32 at a time ------------
    // A group is checked once the stream has passed its last boundary (its
    // bytes are then recent in L2), or at the end of the warp's range.
    while (next_group < b1) {
      const int64_t last = group_last;
      if (t + 1 < t1 && group_last_off >= tile_hi) break;
      const int64_t j = next_group + lane;
      if (j <= last) {
        const int64_t oj = offsets[j];
        if (j >= 1) {  // tail of string j-1, which ends at oj
          const int64_t s = offsets[j - 1];
          const WordLut tail = lut_word(gather4(data, oj - 4, s, oj));
          const uint32_t te = word_error(tail, ascii_lut());  // positions oj .. oj+3
          if (te != 0) charge<LOCATE>(out_valid, out_err, j - 1, oj - s + ((__ffs(te) - 1) >> 3));
        }
        if (j < count) {  // head of string j, which starts at oj
          const int64_t end = offsets[j + 1];
          const WordLut head = lut_word(gather4(data, oj, oj, end));
          const uint32_t he = word_error(ascii_lut(), head);  // positions oj .. oj+3
          if (he != 0) charge<LOCATE>(out_valid, out_err, j, (__ffs(he) - 1) >> 3);
        }
      }
      next_group = last + 1;
      group_last = (next_group + kLanes < b1 ? next_group + kLanes : b1) - 1;
      if (next_group < b1) group_last_off = offsets[group_last];
    }
  }
}

template <int ROWS, bool LOCATE = false>
static cudaError_t launch_batch_rows(const uint8_t* data, const int64_t* offsets, int64_t count,
                                     uint8_t* out_valid, int blocks_per_sm, int sm_count,
                                     cudaStream_t st, utf8_error_info* out_err = nullptr) {
  const unsigned grid = (unsigned)(sm_count * blocks_per_sm);
  batch_kernel<ROWS, LOCATE><<<grid, kBlockThreads, 0, st>>>(data, offsets, count, out_valid,
                                                              out_err);
  return cudaGetLastError();
}

cudaError_t launch_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                         uint8_t* out_valid, const LaunchCfg& cfg, int sm_count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out_valid, 1, (size_t)count, st);
  if (e != cudaSuccess) return e;
  switch (cfg.batch_rows) {
    case 4: return launch_batch_rows<4>(data, offsets, count, out_valid, cfg.batch_blocks_per_sm,
                                        sm_count, st);
    default: return launch_batch_rows<2>(data, offsets, count, out_valid, cfg.batch_blocks_per_sm,
                                         sm_count, st);
  }
}

cudaError_t launch_batch_first_errors(const uint8_t* data, const int64_t* offsets, int64_t count,
                                      utf8_error_info* out, const LaunchCfg& cfg, int sm_count,
                                      cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  switch (cfg.batch_rows) {
    case 4: return launch_batch_rows<4, true>(data, offsets, count, nullptr,
                                              cfg.batch_blocks_per_sm, sm_count, st, out);
    default: return launch_batch_rows<2, true>(data, offsets, count, nullptr,
                                               cfg.batch_blocks_per_sm, sm_count, st, out);
  }
}

}  // namespace utf8gpu

namespace utf8gpu {

int batch_blocks_per_sm(int rows) {
  int n = 0;
  cudaError_t e;
  switch (rows) {
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<4, false>, kBlockThreads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<2, false>, kBlockThreads, 0); break;
  }
  if (e != cudaSuccess) { cudaGetLastError(); return 1; }
  return n > 0 ? n : 1;
}

}  // namespace utf8gpu

// Copy and validate in one pass over HBM.
//
// Ingest pipelines usually copy text into place and then validate it, which
// reads the bytes twice.  copy_kernel streams the source through the same
// tiles and classification as validate_kernel and writes every granule to the
// destination as soon as it is loaded, so the bytes are read once and written
// once.  Source and destination must have the same alignment modulo 16 (then
// granules line up); the first and last granules are written byte by byte so
// nothing outside [dst, dst + len) is touched.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "lookup.cuh"
#include "tiles.cuh"
#include "tune.h"
#include "utf8gpu.h"

namespace utf8gpu {

__device__ __forceinline__ void st_stream(uint8_t* p, const uint4& v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

// Writes the bytes of granule g that lie inside [off, off + n).
__device__ __forceinline__ void store_granule_checked(const Span& s, uint8_t* dst_abase, uint64_t g,
                                                      const uint4& v) {
  const uint64_t base = g * 16;
  const uint64_t end = s.off + s.n;
  if (base >= end || base + 16 <= s.off) return;
  if (base >= s.off && base + 16 <= end) {
    st_stream(dst_abase + base, v);
    return;
  }
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint64_t p = base + k;
    if (p >= s.off && p < end) dst_abase[p] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
  }
}

template <int ROWS>
__global__ void __launch_bounds__(kBlockThreads)
    copy_kernel(Span s, uint8_t* __restrict__ dst_abase, uint64_t tiles, uint8_t* out_valid) {
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
  uint64_t in0, in1;
  interior_tiles<ROWS>(s, in0, in1);
  const uint8_t* lane_ptr = s.abase + t0 * tb + lane * 16;
  uint32_t err = 0;
  uint4 next[ROWS];
  load_tile<ROWS>(s, t0, in0, in1, lane, lane_ptr, next);
  for (uint64_t t = t0; t < t1; ++t, lane_ptr += tb) {
    uint4 d[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) d[r] = next[r];
    if (t + 1 < t1) load_tile<ROWS>(s, t + 1, in0, in1, lane, lane_ptr + tb, next);
    const bool interior = t >= in0 && t < in1;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const uint64_t g = t * TileGeom<ROWS>::kGranules + r * kLanes + lane;
      if (interior) st_stream(dst_abase + g * 16, d[r]);
      else store_granule_checked(s, dst_abase, g, d[r]);
    }
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS>(d, carry, lane, merge_sel, e);
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) err |= e[p][m];
  }
  if (__any_sync(kFull, err != 0) && lane == 0) *out_valid = 0;
}

template <int ROWS>
static cudaError_t launch_copy_rows(const Span& s, uint8_t* dst_abase, uint8_t* out_valid,
                                    int blocks_per_sm, int sm_count, cudaStream_t st) {
  const uint64_t tiles = span_tiles<ROWS>(s);
  const uint64_t warps_per_block = kBlockThreads / kLanes;
  uint64_t grid = (uint64_t)sm_count * (uint64_t)blocks_per_sm;
  const uint64_t need = (tiles + warps_per_block - 1) / warps_per_block;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  copy_kernel<ROWS><<<(unsigned)grid, kBlockThreads, 0, st>>>(s, dst_abase, tiles, out_valid);
  return cudaGetLastError();
}

cudaError_t launch_copy_validate(uint8_t* dst, const uint8_t* src, uint64_t n, uint8_t* out_valid,
                                 const LaunchCfg& cfg, int sm_count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out_valid, 1, 1, st);
  if (e != cudaSuccess || n == 0) return e;
  if ((reinterpret_cast<uintptr_t>(dst) & 15) != (reinterpret_cast<uintptr_t>(src) & 15)) {
    // granules do not line up: copy, then validate the copy (both on the GPU)
    e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return launch_validate_tiles(dst, n, 0, ~uint64_t(0), out_valid, cfg, sm_count, st);
  }
  const Span s = make_span(src, n);
  uint8_t* dst_abase = dst - s.off;
  const int bps = copy_blocks_per_sm(cfg.rows, cfg.blocks_per_sm);
  switch (cfg.rows) {
    case 2: return launch_copy_rows<2>(s, dst_abase, out_valid, bps, sm_count, st);
    case 4: return launch_copy_rows<4>(s, dst_abase, out_valid, bps, sm_count, st);
    default: return launch_copy_rows<8>(s, dst_abase, out_valid, bps, sm_count, st);
  }
}

int copy_blocks_per_sm(int rows, int wanted) {
  int n = 0;
  cudaError_t e;
  switch (rows) {
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, copy_kernel<2>, kBlockThreads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, copy_kernel<4>, kBlockThreads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, copy_kernel<8>, kBlockThreads, 0); break;
  }
  if (e != cudaSuccess) { cudaGetLastError(); n = 1; }
  if (n < 1) n = 1;
  return wanted < n && wanted > 0 ? wanted : n;
}

}  // namespace utf8gpu

// Chunks of a longer stream: the paper's loop carries the previous block
// between iterations and checks the end of the stream once (Section 6,
// Section 6.3); here the carried state is the last three bytes of the stream
// so far, and a chunk is validated exactly as the same bytes would be inside
// the whole stream.
//
// chunk_kernel checks positions [0, n) of a chunk whose previous bytes are
// `prefix` (up to three bytes; zeros at the start of a stream), and, for the
// final chunk, the end-of-stream positions after it.  The prefix bytes are
// inserted into the chunk's virtual layout (before the data, in the first
// granule or in the carry), errors at positions before the chunk are dropped
// (they belong to the previous chunk), and for a non-final chunk so are the
// virtual zero positions after it (the next chunk checks them with its real
// bytes).  One thread also writes the stream's new last three bytes to
// `tail_out` for the next chunk.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "lookup.cuh"
#include "tiles.cuh"
#include "tune.h"

namespace utf8gpu {

struct ChunkArgs {
  uint32_t prefix;           // natural order: byte 3 = b[-1], byte 2 = b[-2], byte 1 = b[-3]
  const uint8_t* prefix_dev;  // if set: b[-3], b[-2], b[-1] read from device memory
  int final_chunk;           // 1: check the end of the stream after this chunk
  uint8_t* out_valid;        // cleared on error, never set
  uint8_t* tail_out;         // if set: receives the new b[-3], b[-2], b[-1]
};

__device__ __forceinline__ uint32_t chunk_prefix(const ChunkArgs& a) {
  if (a.prefix_dev)
    return ((uint32_t)a.prefix_dev[0] << 8) | ((uint32_t)a.prefix_dev[1] << 16) |
           ((uint32_t)a.prefix_dev[2] << 24);
  return a.prefix;
}

// Clears the bytes of the interleaved error words whose virtual position
// (relative to the stream's aligned base) is outside [lo, hi).
template <int ROWS, bool QUADS>
__device__ __forceinline__ void mask_positions(uint32_t (&e)[ROWS / 2][8], uint64_t tile_v,
                                               int lane, uint64_t lo, uint64_t hi) {
#pragma unroll
  for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint64_t v = tile_v + interleaved_position<ROWS, QUADS>(p, m, b, lane);
        if (v < lo || v >= hi) e[p][m] &= ~(0xFFu << (8 * b));
      }
}

constexpr int kChunkRows = 8;       // tile rows per warp (4 KiB tiles), as the single-buffer default
constexpr int kSmallChunkRows = 2;  // 1 KiB tiles for chunks too small to fill the grid

// STAGED (8 rows, where the device gives the rings their shared memory):
// row quads with the tiles through the warp's ring (StagedRun, tiles.cuh);
// otherwise row pairs with register loads (quads with register loads need
// 145 registers, one CTA per SM).
template <int ROWS, bool STAGED = false>
__global__ void __launch_bounds__(kBlockThreads, 2) chunk_kernel(Span s, uint64_t tiles, ChunkArgs a) {
  constexpr bool kQuads = STAGED;
  constexpr uint64_t tb = TileGeom<ROWS>::kBytes;
  const int lane = threadIdx.x & (kLanes - 1);
  const uint64_t warps = (uint64_t)gridDim.x * (kBlockThreads / kLanes);
  const uint64_t w = (uint64_t)blockIdx.x * (kBlockThreads / kLanes) + (threadIdx.x / kLanes);
  const uint32_t pre = chunk_prefix(a);
  if (a.tail_out && blockIdx.x == 0 && threadIdx.x == 0) {
    // new b[-k] (k = 1..3) = data[n - k], or a prefix byte when n < k
    for (int k = 3; k >= 1; --k) {
      const int64_t d = (int64_t)s.n - k;
      const uint8_t v = d >= 0 ? s.abase[s.off + (uint64_t)d] : (uint8_t)(pre >> (8 * (4 + d)));
      a.tail_out[3 - k] = v;
    }
  }
  const uint64_t t0 = tiles * w / warps;
  const uint64_t t1 = tiles * (w + 1) / warps;
  if (t0 >= t1) return;
  const uint32_t merge_sel = carry_merge_selector<kQuads>(lane);
  Carry carry;
  if (t0 == 0) {
    // virtual bytes -4..-1 are data offsets -4-off .. -1-off
    carry = halo_carry<kQuads>(s.off < 4 ? pre << (8 * s.off) : 0u);
  } else {
    carry = halo_carry<kQuads>(load_word(s, t0 * tb - 4));
  }
  const uint64_t keep_hi = a.final_chunk ? ~uint64_t(0) : s.off + s.n;
  uint64_t in0, in1;
  interior_tiles<ROWS>(s, in0, in1);
  const uint8_t* lane_ptr = s.abase + t0 * tb + lane * 16;
  uint32_t err = 0;
  uint4 next[STAGED ? 1 : ROWS];  // register form: the next tile's loads, one tile ahead
  extern __shared__ uint4 chunk_rings[];
  StagedRun<ROWS> ring(s, t0, t1, chunk_rings + (threadIdx.x / kLanes) * kStages * ROWS * kLanes,
                       lane);
  if constexpr (STAGED) ring.start();
  else load_tile<ROWS>(s, t0, in0, in1, lane, lane_ptr, next);
  for (uint64_t t = t0; t < t1; ++t, lane_ptr += tb) {
    uint4 d[ROWS];
    if constexpr (STAGED) {
      ring.next((uint32_t)(t - t0), d);
    } else {
#pragma unroll
      for (int r = 0; r < ROWS; ++r) d[r] = next[r];
      if (t + 1 < t1) load_tile<ROWS>(s, t + 1, in0, in1, lane, lane_ptr + tb, next);
    }
    if (t == 0 && lane == 0) {
      // prefix byte i (data offset i - 4) sits at virtual position off + i - 4
#pragma unroll
      for (int i = 1; i < 4; ++i) {
        const int v = (int)s.off + i - 4;
        const uint32_t add = v >= 0 ? ((pre >> (8 * i)) & 0xFFu) << (8 * (v & 3)) : 0u;
        const int word = v >> 2;
        d[0].x |= word == 0 ? add : 0u;
        d[0].y |= word == 1 ? add : 0u;
        d[0].z |= word == 2 ? add : 0u;
        d[0].w |= word == 3 ? add : 0u;
      }
    }
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS, kQuads>(d, carry, lane, merge_sel, e);
    const uint64_t tile_v = t * tb;
    if (tile_v < s.off || tile_v + tb > keep_hi)
      mask_positions<ROWS, kQuads>(e, tile_v, lane, s.off, keep_hi);
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) err |= e[p][m];
  }
  if constexpr (STAGED) ring.finish();
  if (__any_sync(kFull, err != 0) && lane == 0) *a.out_valid = 0;
}

// Resident CTAs per SM of chunk_kernel<ROWS, STAGED> (the same on every GPU
// of this architecture; computed once, thread-safely).
template <int ROWS, bool STAGED>
static int chunk_blocks_per_sm() {
  static const int n = [] {
    int k = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &k, chunk_kernel<ROWS, STAGED>, kBlockThreads,
            STAGED ? staged_smem_bytes<ROWS>(kBlockThreads) : 0) != cudaSuccess) {
      cudaGetLastError();
      k = 1;
    }
    return k > 0 ? k : 1;
  }();
  return n;
}

template <int ROWS, bool STAGED = false>
static cudaError_t launch_chunk_rows(const Span& s, const ChunkArgs& a, int sm_count,
                                     cudaStream_t st) {
  const uint64_t tiles = span_tiles<ROWS>(s);
  const uint64_t warps_per_block = kBlockThreads / kLanes;
  uint64_t grid = (uint64_t)sm_count * (uint64_t)chunk_blocks_per_sm<ROWS, STAGED>();
  const uint64_t need = (tiles + warps_per_block - 1) / warps_per_block;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  chunk_kernel<ROWS, STAGED>
      <<<(unsigned)grid, kBlockThreads, STAGED ? staged_smem_bytes<ROWS>(kBlockThreads) : 0, st>>>(
          s, tiles, a);
  return cudaGetLastError();
}

cudaError_t prepare_chunk_staged() {
  const int smem = staged_smem_bytes<kChunkRows>(kBlockThreads);
  cudaError_t e = cudaFuncSetAttribute(chunk_kernel<kChunkRows, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chunk_kernel<kChunkRows, true>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t launch_chunk(const uint8_t* data, uint64_t n, uint32_t prefix,
                         const uint8_t* prefix_dev, int final_chunk, uint8_t* out_valid,
                         uint8_t* tail_out, int sm_count, bool staged, cudaStream_t st) {
  const Span s = make_span(data, n);
  const ChunkArgs a{prefix, prefix_dev, final_chunk, out_valid, tail_out};
  // A chunk so small that its 1 KiB tiles number at most the warps of the
  // persistent grid is checked in 1 KiB tiles: 4 KiB tiles would leave SMs
  // idle.
  const uint64_t grid_warps = (uint64_t)sm_count * (uint64_t)chunk_blocks_per_sm<kChunkRows, false>() *
                              (kBlockThreads / kLanes);
  if (span_tiles<kSmallChunkRows>(s) <= grid_warps)
    return launch_chunk_rows<kSmallChunkRows>(s, a, sm_count, st);
  if (staged) return launch_chunk_rows<kChunkRows, true>(s, a, sm_count, st);
  return launch_chunk_rows<kChunkRows>(s, a, sm_count, st);
}

}  // namespace utf8gpu

// ---------------------------------------------------------------------------
// C-ABI: stateless chunks and device-resident stream state
// ---------------------------------------------------------------------------
#include <functional>
#include <mutex>

#include "utf8gpu.h"

using namespace utf8gpu;

namespace {

int status_of(cudaError_t e) {
  if (e != cudaSuccess) cudaGetLastError();
  return set_thread_status(e == cudaSuccess ? UTF8_OK : UTF8_ERR_CUDA);
}

}  // namespace

// Device state: two tail slots (b[-3], b[-2], b[-1]) used alternately, and
// the stream's result byte.
struct utf8_stream {
  uint8_t* dev = nullptr;  // [0..3]: tail slot 0, [4..7]: tail slot 1, [8]: result
  uint64_t chunks = 0;     // non-empty chunks since the last reset
  int sm_count = 0;
  bool staged = false;     // the device's launch configuration stages 8-row tiles
};

extern "C" {

int utf8_validate_chunk(const uint8_t* data, size_t len, uint32_t prefix, int prefix_len,
                        int final_chunk, uint8_t* out_valid, cudaStream_t stream) {
  if (out_valid == nullptr || (data == nullptr && len > 0) || prefix_len < 0 || prefix_len > 3)
    return set_thread_status(UTF8_ERR_INVALID_ARG);
  if (!is_device_memory(out_valid) || (len > 0 && !is_device_memory(data)))
    return set_thread_status(UTF8_ERR_INVALID_ARG);
  const int sms = current_sm_count();
  if (sms <= 0) return set_thread_status(UTF8_ERR_CUDA);
  // prefix byte k (k = 0..2) is b[-1-k]; natural order puts b[-1] in byte 3
  uint32_t pre = 0;
  for (int k = 0; k < prefix_len; ++k) pre |= ((prefix >> (8 * k)) & 0xFFu) << (8 * (3 - k));
  if (len == 0 && !final_chunk) return set_thread_status(UTF8_OK);
  return status_of(launch_chunk(len ? data : out_valid, len, pre, nullptr, final_chunk, out_valid,
                                nullptr, sms, current_config().staged, stream));
}

utf8_stream* utf8_stream_create(void) {
  utf8_stream* s = new utf8_stream();
  s->sm_count = current_sm_count();
  s->staged = current_config().staged;
  cudaError_t e = s->sm_count > 0 ? cudaMalloc(&s->dev, 16) : cudaErrorNoDevice;
  if (e == cudaSuccess) e = cudaMemset(s->dev, 0, 16);
  if (e == cudaSuccess) e = cudaMemset(s->dev + 8, 1, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (s->dev) cudaFree(s->dev);
    delete s;
    set_thread_status(UTF8_ERR_CUDA);
    return nullptr;
  }
  set_thread_status(UTF8_OK);
  return s;
}

int utf8_stream_reset(utf8_stream* s, cudaStream_t stream) {
  if (!s) return set_thread_status(UTF8_ERR_INVALID_ARG);
  s->chunks = 0;
  cudaError_t e = cudaMemsetAsync(s->dev, 0, 8, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->dev + 8, 1, 1, stream);
  return status_of(e);
}

int utf8_stream_update(utf8_stream* s, const uint8_t* chunk, size_t len, cudaStream_t stream) {
  if (!s || (chunk == nullptr && len > 0)) return set_thread_status(UTF8_ERR_INVALID_ARG);
  if (len == 0) return set_thread_status(UTF8_OK);
  if (!is_device_memory(chunk)) return set_thread_status(UTF8_ERR_INVALID_ARG);
  const uint8_t* tail_in = s->dev + 4 * (s->chunks & 1);
  uint8_t* tail_out = s->dev + 4 * ((s->chunks + 1) & 1);
  const cudaError_t e =
      launch_chunk(chunk, len, 0, tail_in, 0, s->dev + 8, tail_out, s->sm_count, s->staged, stream);
  if (e == cudaSuccess) s->chunks += 1;
  return status_of(e);
}

int utf8_stream_finish(utf8_stream* s, uint8_t* out_valid, cudaStream_t stream) {
  if (!s || out_valid == nullptr) return set_thread_status(UTF8_ERR_INVALID_ARG);
  if (!is_device_memory(out_valid)) return set_thread_status(UTF8_ERR_INVALID_ARG);
  // end of stream: an empty final chunk after the current tail
  const uint8_t* tail_in = s->dev + 4 * (s->chunks & 1);
  cudaError_t e = launch_chunk(s->dev + 12, 0, 0, tail_in, 1, s->dev + 8, nullptr, s->sm_count,
                               s->staged, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_valid, s->dev + 8, 1, cudaMemcpyDeviceToDevice, stream);
  return status_of(e);
}

void utf8_stream_destroy(utf8_stream* s) {
  if (!s) return;
  cudaFree(s->dev);
  delete s;
}

}  // extern "C"

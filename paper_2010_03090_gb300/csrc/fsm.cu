// The paper's finite-state validator (Section 5) on the GPU: a comparison
// kernel for the `lookup` path, not the fast path.
//
// Section 5 adapts a decoder's state machine: nine states (valid, 1 / 2 / 3
// more continuation bytes, the four range states after E0, ED, F0 and F4,
// and a sticky error state) and twelve byte classes (ASCII, the three
// continuation ranges 80..8F, 90..9F and A0..BF, and the lead-byte classes),
// one transition per (state, byte); the input is valid iff the machine ends
// in the valid state.  The paper folds the class into a 256-entry table and
// the transition into a 9 x 12 table, notes that a single 9 x 256 table is
// equivalent, and hides the latency of the dependent lookups by running
// three interleaved machines over three regions that each start at a lead
// byte.
//
// Here the 9 x 256 table sits in shared memory (one byte per entry: the next
// state) and every lane runs kInterleave machines over regions of its own.
// The buffer is seen through its 16-byte aligned virtual layout (zero bytes
// before and after the data, as in the other kernels): zeros before the
// data keep the valid state, and the zeros after it turn any unfinished
// character into an error (Section 6.3's end check, for the FSM).  A region
// of kRegionBytes virtual bytes starts after the (at most three) continuation
// bytes at its nominal start; the region before it runs on over them.  So
// every region begins at a character boundary of a valid input, and the
// input is valid exactly when every region ends in the valid state (a fourth
// continuation in a row is met by a machine in the valid state: an error).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tiles.cuh"

namespace utf8gpu {
namespace {

enum FsmState : uint8_t {
  kValid = 0, kOneMore, kTwoMore, kThreeMore,
  kAfterE0,  // 3-byte overlong check: next byte A0..BF
  kAfterED,  // surrogate check: next byte 80..9F
  kAfterF0,  // 4-byte overlong check: next byte 90..BF
  kAfterF4,  // too-large check: next byte 80..8F
  kError,
  kStates
};

// Next state of the machine in state s on byte b (Section 5's transition table).
constexpr uint8_t fsm_next(int s, int b) {
  const bool cont = b >= 0x80 && b <= 0xBF;
  if (s == kError) return kError;
  if (s == kValid) {
    if (b < 0x80) return kValid;
    if (cont || b == 0xC0 || b == 0xC1 || b >= 0xF5) return kError;
    if (b <= 0xDF) return kOneMore;
    if (b == 0xE0) return kAfterE0;
    if (b == 0xED) return kAfterED;
    if (b <= 0xEF) return kTwoMore;
    if (b == 0xF0) return kAfterF0;
    if (b == 0xF4) return kAfterF4;
    return kThreeMore;  // F1..F3
  }
  if (!cont) return kError;  // every other state wants a continuation byte
  switch (s) {
    case kOneMore: return kValid;
    case kTwoMore: return kOneMore;
    case kThreeMore: return kTwoMore;
    case kAfterE0: return b >= 0xA0 ? kOneMore : kError;
    case kAfterED: return b <= 0x9F ? kOneMore : kError;
    case kAfterF0: return b >= 0x90 ? kTwoMore : kError;
    default: return b <= 0x8F ? kTwoMore : kError;  // kAfterF4
  }
}

struct FsmTable {
  uint32_t words[kStates * 256 / 4];  // entry s * 256 + b, packed four per word
};

constexpr FsmTable make_fsm_table() {
  FsmTable t{};
  for (int s = 0; s < kStates; ++s)
    for (int b = 0; b < 256; ++b) {
      const int e = s * 256 + b;
      t.words[e / 4] |= (uint32_t)fsm_next(s, b) << (8 * (e % 4));
    }
  return t;
}

__constant__ FsmTable kFsmTable = make_fsm_table();

constexpr int kRegionBytes = 512;  // nominal region of one machine (a multiple of 16)
constexpr int kInterleave = 4;     // machines per lane
constexpr int kFsmThreads = 256;

// Continuation bytes at the start of word w (bytes 0..2), at most three.
__device__ __forceinline__ uint32_t leading_continuations(uint32_t w) {
  uint32_t k = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const uint32_t b = (w >> (8 * j)) & 0xFFu;
    if ((b & 0xC0u) != 0x80u || k != (uint32_t)j) break;
    k = j + 1;
  }
  return k;
}

// Granule g of the virtual layout, cached in L1: neighbouring granules of a
// machine's region share a 32-byte sector, read one after the other.
__device__ __forceinline__ uint4 fsm_granule(const Span& s, uint64_t g) {
  const uint64_t v = g * 16;
  const uint64_t end = s.off + s.n;
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  if (v >= end || v + 16 <= s.off) return r;
  r = __ldg(reinterpret_cast<const uint4*>(s.abase + v));
  if (v < s.off || v + 16 > end) {
    const int a = v < s.off ? (int)(s.off - v) : 0;
    const int b = (int)(end - v < 16 ? end - v : 16);
    r.x &= keep_bytes(a, b);
    r.y &= keep_bytes(a - 4, b - 4);
    r.z &= keep_bytes(a - 8, b - 8);
    r.w &= keep_bytes(a - 12, b - 12);
  }
  return r;
}

// One step: state q on byte j of word w (the address is q * 256 + byte).
__device__ __forceinline__ uint32_t fsm_step(const uint8_t* tab, uint32_t q, uint32_t w, int j) {
  return tab[prmt(w, q, 0x5540u | (uint32_t)j)];
}

template <int K>
__global__ void __launch_bounds__(kFsmThreads) fsm_kernel(Span s, uint64_t regions,
                                                          uint8_t* out_valid) {
  __shared__ __align__(16) uint32_t tab_words[kStates * 256 / 4];
  for (int i = threadIdx.x; i < kStates * 256 / 4; i += blockDim.x)
    tab_words[i] = kFsmTable.words[i];
  __syncthreads();
  const uint8_t* tab = reinterpret_cast<const uint8_t*>(tab_words);

  const uint64_t threads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  // rounds of K regions per thread: region r = base + k * threads
  for (uint64_t base = t; base < regions; base += threads * K) {
    uint32_t q[K];
    uint32_t skip_end[K];
    uint64_t r0[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t r = base + (uint64_t)k * threads;
      r0[k] = r;
      const uint64_t g0 = r * (kRegionBytes / 16);
      const uint4 first = r < regions ? fsm_granule(s, g0) : make_uint4(0u, 0u, 0u, 0u);
      const uint4 next = r + 1 < regions ? fsm_granule(s, g0 + kRegionBytes / 16)
                                         : make_uint4(0u, 0u, 0u, 0u);
      // the region starts after the continuations at its nominal start (not
      // the first region: there they are an error the machine finds)
      const uint32_t skip = r == 0 || r >= regions ? 0u : leading_continuations(first.x);
      skip_end[k] = leading_continuations(next.x);
      uint32_t st = kValid;
      const uint32_t w[4] = {first.x, first.y, first.z, first.w};
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if ((uint32_t)j >= skip) st = fsm_step(tab, st, w[j >> 2], j & 3);
      q[k] = r < regions ? st : (uint32_t)kValid;
    }
    // interior granules: K machines side by side
    for (int g = 1; g < kRegionBytes / 16; ++g) {
      uint4 v[K];
#pragma unroll
      for (int k = 0; k < K; ++k)
        v[k] = r0[k] < regions ? fsm_granule(s, r0[k] * (kRegionBytes / 16) + g)
                               : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int j = 0; j < 16; ++j)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const uint32_t w = j < 4 ? v[k].x : j < 8 ? v[k].y : j < 12 ? v[k].z : v[k].w;
          q[k] = fsm_step(tab, q[k], w, j & 3);
        }
    }
    // run on over the next region's leading continuations; the last region
    // of the stream also sees its trailing zeros (within its own granules)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (r0[k] >= regions) continue;
      const uint64_t gn = (r0[k] + 1) * (kRegionBytes / 16);
      const uint4 nx = r0[k] + 1 < regions ? fsm_granule(s, gn) : make_uint4(0u, 0u, 0u, 0u);
      uint32_t st = q[k];
      for (uint32_t j = 0; j < skip_end[k]; ++j) st = fsm_step(tab, st, nx.x, (int)j);
      bad |= st != kValid;
    }
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & (kLanes - 1)) == 0) clear_result(out_valid);
}

}  // namespace

// One buffer through the finite-state machine; out_valid must hold 1 before
// the launch (cleared on an error).
cudaError_t launch_validate_fsm(const uint8_t* data, uint64_t n, uint8_t* out_valid, int sm_count,
                                cudaStream_t st) {
  const Span s = make_span(data, n);
  const uint64_t regions = (s.granules * 16 + kRegionBytes - 1) / kRegionBytes;
  const uint64_t need = (regions + (uint64_t)kInterleave * kFsmThreads - 1) /
                        ((uint64_t)kInterleave * kFsmThreads);
  uint64_t grid = (uint64_t)sm_count * 8;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  fsm_kernel<kInterleave><<<(unsigned)grid, kFsmThreads, 0, st>>>(s, regions, out_valid);
  return cudaGetLastError();
}

}  // namespace utf8gpu

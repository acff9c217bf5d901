// Warp-level streaming of one byte range through the `lookup` checks.
//
// A stream (a whole buffer, or one string of a batch) is seen through its
// 16-byte aligned "virtual" layout: virtual byte v is abase[v] when
// off <= v < off + n and 0 otherwise, where abase = data rounded down to 16
// bytes and off = data - abase.  The zeros before `off` are the paper's zero
// previous block at the start of a stream (Section 6); the (at least three)
// zeros after off + n are the ASCII padding that makes the end-of-stream
// check (Section 6.3) part of the ordinary classification.
//
// A tile is ROWS rows of GROUP lanes x 16 bytes: row r of tile t is the
// contiguous GROUP*16 bytes at granule (t*ROWS + r)*GROUP, so every load
// instruction of a group reads contiguous bytes (512 for a whole warp).  Byte
// i's previous bytes come from the same lane, from the lane to the left (a
// shuffle of that lane's last-word lookups) or, for the group's first lane,
// from the previous row (carried in registers).  A warp starting in the middle
// of a stream first reads the 4 bytes before its first tile (the halo).
//
// Only aligned 16-byte granules holding at least one byte of [off, off + n)
// are read, so no access leaves the pages of the caller's buffer.
#pragma once
#include <stdint.h>
#include "lookup.cuh"

namespace utf8gpu {

constexpr int kLanes = 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct Span {
  const uint8_t* abase;  // 16-byte aligned
  uint64_t off;          // data - abase, 0..15
  uint64_t n;            // bytes in the stream
  uint64_t granules;     // ceil((off + n + 3) / 16): data plus three zero bytes
};

__host__ __device__ inline Span make_span(const uint8_t* data, uint64_t n) {
  Span s;
  const uintptr_t p = reinterpret_cast<uintptr_t>(data);
  s.abase = reinterpret_cast<const uint8_t*>(p & ~uintptr_t(15));
  s.off = p & 15;
  s.n = n;
  s.granules = (s.off + n + 3 + 15) / 16;
  return s;
}

template <int ROWS, int GROUP = 32>
__host__ __device__ inline uint64_t span_tiles(const Span& s) {
  return (s.granules + (uint64_t)GROUP * ROWS - 1) / ((uint64_t)GROUP * ROWS);
}

// Streaming 16-byte load: read once, do not keep in L1.
__device__ __forceinline__ uint4 ld_stream(const uint8_t* p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

// Mask keeping the bytes of a word whose index (0..3) lies in [a, b).
__device__ __forceinline__ uint32_t keep_bytes(int a, int b) {
  a = a < 0 ? 0 : a;
  b = b > 4 ? 4 : b;
  if (b <= a) return 0u;
  return (uint32_t)((((uint64_t)1 << (8 * (b - a))) - 1) << (8 * a));
}

// Granule g of the virtual layout.
__device__ __forceinline__ uint4 load_granule(const Span& s, uint64_t g) {
  const uint64_t v = g * 16;
  const uint64_t end = s.off + s.n;
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  if (v >= end || v + 16 <= s.off) return r;  // no byte of the data: nothing to read
  r = ld_stream(s.abase + v);
  if (v < s.off || v + 16 > end) {  // first or last granule of the stream
    const int a = v < s.off ? (int)(s.off - v) : 0;
    const int b = (int)(end - v < 16 ? end - v : 16);
    r.x &= keep_bytes(a, b);
    r.y &= keep_bytes(a - 4, b - 4);
    r.z &= keep_bytes(a - 8, b - 8);
    r.w &= keep_bytes(a - 12, b - 12);
  }
  return r;
}

// The 4 virtual bytes [v, v + 4) (v a multiple of 4), zero outside the data.
__device__ __forceinline__ uint32_t load_word(const Span& s, uint64_t v) {
  const uint64_t end = s.off + s.n;
  if (v + 4 <= s.off || v >= end) return 0u;
  const uint32_t w = *reinterpret_cast<const uint32_t*>(s.abase + v);
  const int a = v < s.off ? (int)(s.off - v) : 0;
  const int b = (int)(end - v < 4 ? end - v : 4);
  return w & keep_bytes(a, b);
}

template <int GROUP>
__device__ __forceinline__ WordLut shfl_lut(const WordLut& l, int src) {
  WordLut r;
  r.prev_side = __shfl_sync(kFull, l.prev_side, src, GROUP);
  r.cur_side = 0;  // a left neighbour only ever serves as "previous"
  r.flags = __shfl_sync(kFull, l.flags, src, GROUP);
  return r;
}

// Checks tiles [t_begin, t_end) of a stream with a group of GROUP lanes
// (GROUP = 8, 16 or 32; the 32 / GROUP groups of a warp each have their own
// stream and range).  A tile is ROWS rows of GROUP lanes x 16 bytes.  All
// groups run `trip` iterations (trip >= t_end - t_begin of every group) so
// that warp-wide shuffles and votes stay converged; a group whose range is
// exhausted idles.  Returns a non-zero value in some lane of the group iff
// an error lies in the group's tiles.  Call with the whole warp.
template <int ROWS, int GROUP>
__device__ __forceinline__ uint32_t group_check_tiles(const Span& s, uint64_t t_begin,
                                                      uint64_t t_end, uint64_t trip) {
  constexpr uint64_t kTileGranules = (uint64_t)GROUP * ROWS;
  const int lane = threadIdx.x & (kLanes - 1);
  const int glane = lane & (GROUP - 1);
  const int left = (glane + GROUP - 1) & (GROUP - 1);
  const unsigned gmask = GROUP == 32 ? kFull : (((1u << GROUP) - 1u) << (lane & ~(GROUP - 1)));
  uint32_t err = 0;
  WordLut carry = ascii_lut();  // lookups of the 4 bytes before the row (group lane 0)
  if (t_begin < t_end && t_begin > 0)
    carry = lut_word(load_word(s, t_begin * kTileGranules * 16 - 4));

  for (uint64_t i = 0; i < trip; ++i) {
    const uint64_t t = t_begin + i;
    const bool active = t < t_end;
    const uint64_t g0 = t * kTileGranules;
    uint4 d[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
      d[r] = active ? load_granule(s, g0 + r * GROUP + glane) : make_uint4(0u, 0u, 0u, 0u);

    uint32_t high = 0;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) high |= d[r].x | d[r].y | d[r].z | d[r].w;
    const unsigned nonascii = __ballot_sync(kFull, (high & 0x80808080u) != 0);
    if ((nonascii & gmask) == 0) {
      // All-ASCII tile (Section 6.4): no classification, but the bytes before
      // the tile must not end inside a character.
      if (active && glane == 0) err |= word_error(carry, lut_word(d[0].x));
      carry = ascii_lut();
    }
    // The classification runs when any group of the warp needs it; a group
    // whose tile is ASCII (or idle) computes on its own bytes, harmlessly.
    if (nonascii != 0) {
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        WordLut l0, l1, l2, l3;
        lut_pair(d[r].x, d[r].y, l0, l1);
        lut_pair(d[r].z, d[r].w, l2, l3);
        const WordLut from_left = shfl_lut<GROUP>(l3, left);  // group lane 0 gets the last lane
        WordLut prev = from_left;
        if (glane == 0) prev = carry;
        const uint32_t e =
            word_error(prev, l0) | word_error(l0, l1) | word_error(l1, l2) | word_error(l2, l3);
        const bool live = active && (nonascii & gmask) != 0 && g0 + r * GROUP < s.granules;
        if (live) {
          err |= e;
          carry = from_left;
        }
      }
    }
  }
  return err;
}

template <int ROWS>
__device__ __forceinline__ uint32_t warp_check_tiles(const Span& s, uint64_t t_begin,
                                                     uint64_t t_end) {
  return group_check_tiles<ROWS, 32>(s, t_begin, t_end, t_end > t_begin ? t_end - t_begin : 0);
}

}  // namespace utf8gpu

// Error location: from the first erroneous position of the `lookup`
// classification to the length of the longest valid prefix and the Section 3
// rule that the next character breaks.
//
// The classification (Section 6) gives an error byte per position i, computed
// from bytes i-3 .. i.  Let L be the longest valid prefix.  Every position
// before L is clean, and the character starting at L shows an error at L (a
// stray continuation, or a lead with too few continuations at the end), at L+1
// (the second-byte checks of Table 7), or where a continuation byte is
// missing (at most L+3, or an end-of-stream position up to n+2).  So the
// first erroneous position p lies in [L, L+3].  For m <= p every position
// before m is clean, so data[0 .. m) is valid exactly when no character is cut
// at m: the end-of-stream check of Section 6.3 (none of the last three bytes
// starts a character longer than the bytes left).  L is therefore the last
// m <= min(p, n) at which no character is cut, at most three steps back.
#pragma once
#include <stdint.h>

#include "tiles.cuh"
#include "utf8gpu.h"

namespace utf8gpu {

constexpr unsigned long long kNoError = ~0ull;

// Smallest tile-relative position of a non-zero error byte in this lane's
// interleaved error words (see check_tile); 0xFFFFFFFF if there is none.
template <int ROWS>
__device__ __forceinline__ uint32_t lane_first_error(const uint32_t (&e)[ROWS / 2][8], int lane) {
  uint32_t best = 0xFFFFFFFFu;
#pragma unroll
  for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      uint32_t bits = e[p][m];
      while (bits != 0) {
        const int byte = (__ffs(bits) - 1) >> 3;
        bits &= ~(0xFFu << (8 * byte));
        const uint32_t v = interleaved_position<ROWS>(p, m, byte, lane);
        best = v < best ? v : best;
      }
    }
  return best;
}

// Section 6.3's end check on the prefix s[0 .. m): no character is cut at m.
__device__ __forceinline__ bool whole_characters_before(const uint8_t* s, uint64_t m) {
  const uint32_t c1 = m >= 1 ? s[m - 1] : 0u;
  const uint32_t c2 = m >= 2 ? s[m - 2] : 0u;
  const uint32_t c3 = m >= 3 ? s[m - 3] : 0u;
  return !(c1 >= 0xC0u || c2 >= 0xE0u || c3 >= 0xF0u);
}

// The Section 3 rule (a-f as 1-6) broken by the character at c[0], with len
// bytes available: header bits first, then each continuation byte, then the
// decoded code point.
__device__ __forceinline__ int32_t broken_rule(const uint8_t* c, uint64_t len) {
  if (len == 0) return UTF8_RULE_NONE;
  const uint32_t lead = c[0];
  if (lead < 0x80u) return UTF8_RULE_NONE;  // an ASCII byte is a whole character
  if (lead < 0xC0u) return UTF8_RULE_TOO_LONG;
  if (lead >= 0xF8u) return UTF8_RULE_5PLUS_BYTE;
  const int k = lead >= 0xF0u ? 4 : lead >= 0xE0u ? 3 : 2;
  uint32_t cp = lead & (0x7Fu >> k);
  for (int i = 1; i < k; ++i) {
    if ((uint64_t)i >= len || (c[i] & 0xC0u) != 0x80u) return UTF8_RULE_TOO_SHORT;
    cp = (cp << 6) | (c[i] & 0x3Fu);
  }
  if (cp < (k == 2 ? 0x80u : k == 3 ? 0x800u : 0x10000u)) return UTF8_RULE_OVERLONG;
  if (cp > 0x10FFFFu) return UTF8_RULE_TOO_LARGE;
  if (cp >= 0xD800u && cp <= 0xDFFFu) return UTF8_RULE_SURROGATE;
  return UTF8_RULE_NONE;
}

// Turns the first erroneous position p of s[0 .. n) (kNoError if none) into
// the error location.
__device__ __forceinline__ void settle_location(const uint8_t* s, uint64_t n,
                                                unsigned long long p, utf8_error_info* out) {
  if (p == kNoError) {
    out->position = n;
    out->rule = UTF8_RULE_NONE;
    out->reserved = 0;
    return;
  }
  uint64_t m = p < n ? p : n;
  for (int k = 0; k < 3 && !whole_characters_before(s, m); ++k) --m;
  out->position = m;
  out->rule = broken_rule(s + m, n - m);
  out->reserved = 0;
}

// The position field as other warps of the grid leave it (GPU-scope relaxed
// load, ordered with their atomic minima).
__device__ __forceinline__ uint64_t load_position(const utf8_error_info* out) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&out->position));
  return v;
}

// Atomic minimum on a location's position field (set to all ones beforehand).
__device__ __forceinline__ void mark_first_error(utf8_error_info* out, uint64_t position) {
  atomicMin(reinterpret_cast<unsigned long long*>(&out->position),
            (unsigned long long)position);
}

}  // namespace utf8gpu

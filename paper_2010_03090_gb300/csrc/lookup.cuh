// Device-side `lookup` classification (Keiser & Lemire, Section 6).
//
// The paper classifies every byte with three 16-entry tables, indexed by the
// high nibble and the low nibble of the previous byte and the high nibble of
// the current byte, AND-ed together (Section 6.1, Fig. 1, Table 7); it then
// compares bit 7 (two continuations in a row) with the positions where a
// 3- or 4-byte lead two or three bytes back requires one (Section 6.2), and
// pads the end of the stream with ASCII zeros (Section 6.3).  Any non-zero
// byte of  (byte_1_high & byte_1_low & byte_2_high) ^ must_be_2_3  is an error.
//
// On the GPU the 16-byte shuffle of the paper (vpshufb / tbl) becomes the
// byte-permute instruction `prmt`, four lookups per 32-bit word, with these
// design points (all exact; an exhaustive test over every byte pair and every
// (prev3, prev2) pair checks them against the tables):
//
//  * Nibble selectors.  prmt takes four 4-bit selectors packed in 16 bits.
//    In the streaming kernels two rows of a tile are processed side by side
//    (lut_interleaved): interleaving their bytes lets one shift and one mask
//    pack the selectors of eight bytes.
//  * 16 entries from an 8-byte prmt table.  A selector nibble with bit 3 set
//    makes prmt replicate the sign bit of the selected byte.  With the
//    complemented high nibble (15 - n) the eight non-ASCII leads 8..F index
//    an ordinary 8-byte table; ASCII bytes fall into sign mode and are
//    replaced afterwards by the table's constant for 0..7 (0x02 for
//    byte_1_high, 0x01 for byte_2_high), under a mask of the bytes' sign bits.
//  * byte_1_low has bit 7 set in all 16 entries, so a lookup through the
//    plain low nibble (entries 0..7, sign mode gives 0xFF for 8..F) AND-ed
//    with a lookup through the complemented low nibble (entries 8..F, 0xFF for
//    0..7) gives the table exactly.
//  * The previous-byte lookups are computed on the current bytes, then moved
//    to the next position by a funnel shift (the paper's prev<1>), so each
//    byte is looked up once.
//  * must_be_2_3: one more high-nibble lookup gives bit 6 = (byte >= 0xE0)
//    and bit 5 = (byte >= 0xF0); shifts move bit 6 of the byte two back and
//    bit 5 of the byte three back onto bit 7, and their OR under 0x80808080
//    is the paper's (prev2 >= 0xE0) | (prev3 >= 0xF0) mask.
//
// Bit assignment: the one printed in Table 8 (TOO_SHORT 0x01, TOO_LONG 0x02,
// OVERLONG_3 0x04, TOO_LARGE 0x08, SURROGATE 0x10, OVERLONG_2 0x20,
// OVERLONG_4 | TOO_LARGE_1000 0x40, TWO_CONTS 0x80).
#pragma once
#include <stdint.h>

namespace utf8gpu {

// ---------------------------------------------------------------------------
// The three tables of Section 6.1, entry n = nibble value n (Table 8 values).
// ---------------------------------------------------------------------------
constexpr uint8_t kByte1High[16] = {
    0x02, 0x02, 0x02, 0x02, 0x02, 0x02, 0x02, 0x02,   // 0xxx: ASCII -> TOO_LONG
    0x80, 0x80, 0x80, 0x80,                           // 10xx: continuation
    0x21,                                             // 1100: TOO_SHORT | OVERLONG_2
    0x01,                                             // 1101: TOO_SHORT
    0x15,                                             // 1110: TOO_SHORT | OVERLONG_3 | SURROGATE
    0x49};                                            // 1111: TOO_SHORT | TOO_LARGE | 0x40
constexpr uint8_t kByte1Low[16] = {
    0xE7, 0xA3, 0x83, 0x83, 0x8B, 0xCB, 0xCB, 0xCB,
    0xCB, 0xCB, 0xCB, 0xCB, 0xCB, 0xDB, 0xCB, 0xCB};
constexpr uint8_t kByte2High[16] = {
    0x01, 0x01, 0x01, 0x01, 0x01, 0x01, 0x01, 0x01,   // ASCII: TOO_SHORT
    0xE6, 0xAE, 0xBA, 0xBA,                           // continuations
    0x01, 0x01, 0x01, 0x01};                          // leads: TOO_SHORT
// must_be_2_3 flags per high nibble: bit 6 = (byte >= 0xE0), bit 5 = (byte >= 0xF0)
constexpr uint8_t kLeadFlags[16] = {
    0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0x40, 0x60};

constexpr uint32_t kTwoConts = 0x80808080u;

constexpr uint32_t pack4(uint8_t b0, uint8_t b1, uint8_t b2, uint8_t b3) {
  return (uint32_t)b0 | ((uint32_t)b1 << 8) | ((uint32_t)b2 << 16) | ((uint32_t)b3 << 24);
}
// entries 0..7 as an 8-byte prmt table (plain selector)
constexpr uint32_t lowHalf(const uint8_t* t, int w) {
  return pack4(t[4 * w], t[4 * w + 1], t[4 * w + 2], t[4 * w + 3]);
}
// entries 15..8 as an 8-byte prmt table (complemented selector: slot k = 15 - n)
constexpr uint32_t highHalfReversed(const uint8_t* t, int w) {
  return pack4(t[15 - 4 * w], t[14 - 4 * w], t[13 - 4 * w], t[12 - 4 * w]);
}

constexpr uint32_t kB1H_R0 = highHalfReversed(kByte1High, 0), kB1H_R1 = highHalfReversed(kByte1High, 1);
constexpr uint32_t kB2H_R0 = highHalfReversed(kByte2High, 0), kB2H_R1 = highHalfReversed(kByte2High, 1);
constexpr uint32_t kFlg_R0 = highHalfReversed(kLeadFlags, 0), kFlg_R1 = highHalfReversed(kLeadFlags, 1);
constexpr uint32_t kB1L_L0 = lowHalf(kByte1Low, 0), kB1L_L1 = lowHalf(kByte1Low, 1);
constexpr uint32_t kB1L_R0 = highHalfReversed(kByte1Low, 0), kB1L_R1 = highHalfReversed(kByte1Low, 1);
constexpr uint32_t kAsciiB1H = 0x01010101u * kByte1High[0];
constexpr uint32_t kAsciiB2H = 0x01010101u * kByte2High[0];

static_assert(kFlg_R1 == 0 && (kFlg_R0 & 0x80808080u) == 0,
              "lead flags must stay clear of bit 7 so ASCII sign-mode lookups give 0");
static_assert((kB1L_L0 & kB1L_L1 & kB1L_R0 & kB1L_R1 & 0x80808080u) == 0x80808080u,
              "byte_1_low must have bit 7 in every entry for the AND merge");
static_assert((kB1L_L0 & kB1L_L1 & kB1L_R0 & kB1L_R1 & kAsciiB1H) == kAsciiB1H,
              "for an ASCII previous byte, byte_1_high & byte_1_low is byte_1_high's 0x02");

// ---------------------------------------------------------------------------
// primitives
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// Bit select (a & m) | (b & ~m), and its complement, as one three-input LOP3
// each.  Written as C with the two masks 0x0F0F0F0F and 0xF0F0F0F0 the
// compiler sees four operands and emits two LOP3 per select (ncu opcode
// counts: 6 instead of 3 for the selectors of a word pair).
__device__ __forceinline__ uint32_t bit_select(uint32_t a, uint32_t b, uint32_t m) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(a), "r"(b), "r"(m));
  return d;
}
__device__ __forceinline__ uint32_t bit_select_not(uint32_t a, uint32_t b, uint32_t m) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x1B;" : "=r"(d) : "r"(a), "r"(b), "r"(m));
  return d;
}

// Lookup results for one 32-bit word (four consecutive bytes).
struct WordLut {
  uint32_t prev_side;  // byte_1_high[hi] & byte_1_low[lo] of each byte (used as prev1)
  uint32_t cur_side;   // byte_2_high[hi] of each byte
  uint32_t flags;      // bit 6: byte >= 0xE0, bit 5: byte >= 0xF0
};

// Table lookups for one word, given its packed selectors.
//   nonascii : 0xFF in each byte whose byte value has its msb set
//   hi_c     : complemented high nibbles in bits 0..15
//   lo, lo_c : low nibbles and their complements in bits 0..15
__device__ __forceinline__ WordLut lut_from_selectors(uint32_t nonascii, uint32_t hi_c, uint32_t lo,
                                                      uint32_t lo_c) {
  const uint32_t b1h = prmt(kB1H_R0, kB1H_R1, hi_c);
  const uint32_t b2h = prmt(kB2H_R0, kB2H_R1, hi_c);
  const uint32_t b1l = prmt(kB1L_L0, kB1L_L1, lo) & prmt(kB1L_R0, kB1L_R1, lo_c);
  WordLut r;
  r.prev_side = ((b1h & b1l) & nonascii) | (kAsciiB1H & ~nonascii);
  r.cur_side = (b2h & nonascii) | (kAsciiB2H & ~nonascii);
  r.flags = prmt(kFlg_R0, kFlg_R1, hi_c);
  return r;
}

// Lookups for two consecutive words c (bytes 0..3) and d (bytes 4..7), results
// in natural byte order.
__device__ __forceinline__ void lut_pair(uint32_t c, uint32_t d, WordLut& lc, WordLut& ld) {
  const uint32_t u = prmt(c, d, 0x6420);  // c0 c2 d0 d2
  const uint32_t v = prmt(c, d, 0x7531);  // c1 c3 d1 d3
  // nibble k of the selector = nibble of byte k (k = 0..3 for c, 4..7 for d)
  const uint32_t lo_mask = 0x0F0F0F0Fu;
  const uint32_t hi_c = bit_select_not(u >> 4, v, lo_mask);
  const uint32_t lo = bit_select(u, v << 4, lo_mask);
  const uint32_t lo_c = bit_select_not(u, v << 4, lo_mask);
  lc = lut_from_selectors(prmt(c, 0, 0xBA98), hi_c, lo, lo_c);
  ld = lut_from_selectors(prmt(d, 0, 0xBA98), hi_c >> 16, lo >> 16, lo_c >> 16);
}

// Lookups for a single word (halo words, boundary checks and the debug path).
__device__ __forceinline__ WordLut lut_word(uint32_t c) {
  WordLut a, b;
  lut_pair(c, 0, a, b);
  return a;
}

// Lookups for word c of one stream and word d of another, interleaved:
//   A = (c0, d0, c1, d1), B = (c2, d2, c3, d3).
// With two streams side by side a single shift and mask packs the nibble
// selectors of eight bytes, and the previous bytes of a word are a 16-bit
// funnel shift (prev1), the previous word itself (prev2) or a 16-bit funnel
// of the two previous words (prev3).
__device__ __forceinline__ void lut_interleaved(uint32_t c, uint32_t d, WordLut& A, WordLut& B) {
  // nibble k of the selectors: the high / low nibble of byte k of (c0, d0, c1, d1, ...)
  const uint32_t lo_mask = 0x0F0F0F0Fu;
  const uint32_t hi_c = bit_select_not(c >> 4, d, lo_mask);
  const uint32_t lo = bit_select(c, d << 4, lo_mask);
  const uint32_t lo_c = bit_select_not(c, d << 4, lo_mask);
  A = lut_from_selectors(prmt(c, d, 0xD9C8), hi_c, lo, lo_c);
  B = lut_from_selectors(prmt(c, d, 0xFBEA), hi_c >> 16, lo >> 16, lo_c >> 16);
}

// special_cases (Fig. 1) for the four bytes of a word, given the previous
// word's lookups: prev1 = previous byte.
__device__ __forceinline__ uint32_t special_cases(const WordLut& prev, const WordLut& cur) {
  return __funnelshift_l(prev.prev_side, cur.prev_side, 8) & cur.cur_side;
}

// must_be_2_3_continuation (Section 6.2) for the four bytes of a word.
__device__ __forceinline__ uint32_t must_be_2_3(const WordLut& prev, const WordLut& cur) {
  return (__funnelshift_l(prev.flags, cur.flags, 17) | __funnelshift_l(prev.flags, cur.flags, 26)) &
         kTwoConts;
}

// Non-zero iff one of the word's four positions is an error (natural order).
__device__ __forceinline__ uint32_t word_error(const WordLut& prev, const WordLut& cur) {
  return special_cases(prev, cur) ^ must_be_2_3(prev, cur);
}

// The same for an interleaved word W_m, given W_{m-1} (p1) and W_{m-2} (p2):
// prev1 = funnel(W_{m-1}, W_m, 16); prev2 = W_{m-1} (flag bit 6 -> bit 7);
// prev3 = funnel(W_{m-2}, W_{m-1}, 16) (flag bit 5 -> bit 7, so 18 bits).
__device__ __forceinline__ uint32_t interleaved_error(const WordLut& p2, const WordLut& p1,
                                                      const WordLut& cur) {
  const uint32_t sc = __funnelshift_l(p1.prev_side, cur.prev_side, 16) & cur.cur_side;
  const uint32_t m = ((p1.flags << 1) | __funnelshift_l(p2.flags, p1.flags, 18)) & kTwoConts;
  return sc ^ m;
}

// Lookups of an all-ASCII word (also the zero padding before a stream).
__device__ __forceinline__ WordLut ascii_lut() {
  WordLut r;
  r.prev_side = kAsciiB1H;  // byte_1_high & byte_1_low of an ASCII byte: TOO_LONG only
  r.cur_side = kAsciiB2H;
  r.flags = 0;
  return r;
}

}  // namespace utf8gpu

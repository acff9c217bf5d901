// Device-side `lookup` classification (Keiser & Lemire, Section 6).
//
// The paper classifies every byte with three 16-entry tables, indexed by the
// high nibble and the low nibble of the previous byte and the high nibble of
// the current byte, AND-ed together (Section 6.1, Fig. 1, Table 7); it then
// compares bit 7 (two continuations in a row) with the positions where a
// 3- or 4-byte lead two or three bytes back requires one (Section 6.2), and
// pads the end of the stream with ASCII zeros (Section 6.3).
//
// On the GPU the 16-byte shuffle of the paper (vpshufb / tbl) becomes the
// byte-permute instruction `prmt`, four lookups per 32-bit word.  prmt takes
// four 4-bit selectors; a selector with bit 3 set does not look up an entry
// but replicates the sign bit of byte (selector & 7).  With the complemented
// high nibble (15 - n) as selector, the eight non-ASCII high nibbles 8..F
// index an ordinary 8-byte table and every ASCII byte comes out as 0x00 or
// 0xFF, set by the sign bits of that table.  The classification is arranged
// so that those sign-mode values are the right ones, with no per-byte
// correction for ASCII:
//
//  * The five second-byte rows of Table 7 (OVERLONG_2, OVERLONG_3,
//    SURROGATE, TOO_LARGE, OVERLONG_4 | TOO_LARGE_1000) keep the paper's
//    three AND-ed tables, one bit each.  byte_1_high has bit 7 in every
//    non-ASCII entry, so an ASCII previous byte reads 0xFF: it then matches a
//    special row only together with a continuation after it, a pair that is
//    invalid anyway.  byte_2_high has no bit 7 anywhere, so an ASCII current
//    byte reads 0x00 and matches nothing.
//  * The other three rows of Table 7 (TOO_SHORT: a lead not followed by a
//    continuation; TOO_LONG: a continuation after ASCII; TWO_CONTS, checked
//    against must_be_2_3) all say one thing: byte i is a continuation exactly
//    when one is expected there, i.e. when byte i-1 >= 0xC0, byte i-2 >= 0xE0
//    or byte i-3 >= 0xF0.  Section 6.2 builds the last two terms
//    (must_be_2_3); the first is the TOO_SHORT / TOO_LONG pair.  Here the
//    whole condition is one bit (0x40): the current side's table sets it for
//    continuations, the previous side's tables set it for every byte, and the
//    expectation is XOR-ed onto it, so bit 6 of a position is non-zero iff
//    "is a continuation" differs from "expects one".  The expectation comes
//    from a fourth lookup of lead flags (bit 6: >= 0xC0, bit 5: >= 0xE0,
//    bit 4: >= 0xF0), moved onto bit 6 from one, two and three bytes back.
//  * byte_1_low has bit 7 in all 16 entries, so a lookup through the plain
//    low nibble (entries 0..7, sign mode gives 0xFF for 8..F) AND-ed with a
//    lookup through the complemented low nibble (entries 8..F, 0xFF for 0..7)
//    gives the table exactly.
//  * The previous-byte lookups are computed on the current bytes and used at
//    the next position (the paper's prev<1>), so each byte is looked up once.
//    The kernels classify four rows of a tile side by side, one byte of each
//    row per word (lut_quad): the previous bytes of a word are then the
//    previous word itself, with no shift at all.  Two rows side by side
//    (lut_interleaved) need a 16-bit funnel shift.
//
// A position is an error iff its byte  ((prev side of byte i-1) & (current
// side of byte i)) ^ (expectation of byte i)  is non-zero; it has no bits
// outside 0x5F.  This decides exactly the paper's boolean: an exhaustive test
// checks the tables against Table 7's rows (the special bits equal the
// paper's wherever the previous byte is not ASCII) and the whole check
// against the oracle on every class string of up to six bytes.
#pragma once
#include <stdint.h>

namespace utf8gpu {

// ---------------------------------------------------------------------------
// Bits of a position's classification byte.
// ---------------------------------------------------------------------------
constexpr uint8_t kOverlong2 = 0x01;  // C0, C1 + continuation            (Table 7: OVERLONG_2)
constexpr uint8_t kOverlong3 = 0x02;  // E0 + 80..9F                      (OVERLONG_3)
constexpr uint8_t kSurrogate = 0x04;  // ED + A0..BF                      (SURROGATE)
constexpr uint8_t kTooLarge = 0x08;   // F4..FF + 90..BF                  (TOO_LARGE)
constexpr uint8_t kOverlong4 = 0x10;  // F0, F5..FF + 80..8F  (OVERLONG_4 | TOO_LARGE_1000)
constexpr uint8_t kCont = 0x40;       // continuation (current side; every previous byte)
constexpr uint8_t kSpecialBits = 0x1F;
constexpr uint32_t kContBits = 0x40404040u;
// lead flags (current byte): kCont = >= 0xC0, 0x20 = >= 0xE0, 0x10 = >= 0xF0
constexpr uint8_t kGeE0 = 0x20, kGeF0 = 0x10;

// The tables, entry n = nibble value n.
// byte_1_high: entries 0..7 are what prmt's sign mode produces for ASCII.
constexpr uint8_t kByte1High[16] = {
    0xFF, 0xFF, 0xFF, 0xFF, 0xFF, 0xFF, 0xFF, 0xFF,    // ASCII (sign mode)
    0xC0, 0xC0, 0xC0, 0xC0,                            // continuation
    0xC0 | kOverlong2,                                 // 1100
    0xC0,                                              // 1101
    0xC0 | kOverlong3 | kSurrogate,                    // 1110
    0xC0 | kTooLarge | kOverlong4};                    // 1111
constexpr uint8_t kByte1Low[16] = {
    0xC0 | kOverlong2 | kOverlong3 | kOverlong4,       // 0
    0xC0 | kOverlong2,                                 // 1
    0xC0, 0xC0,                                        // 2, 3
    0xC0 | kTooLarge,                                  // 4
    0xC0 | kTooLarge | kOverlong4, 0xC0 | kTooLarge | kOverlong4,
    0xC0 | kTooLarge | kOverlong4, 0xC0 | kTooLarge | kOverlong4,
    0xC0 | kTooLarge | kOverlong4, 0xC0 | kTooLarge | kOverlong4,
    0xC0 | kTooLarge | kOverlong4, 0xC0 | kTooLarge | kOverlong4,    // 5..C
    0xC0 | kTooLarge | kOverlong4 | kSurrogate,                      // D
    0xC0 | kTooLarge | kOverlong4, 0xC0 | kTooLarge | kOverlong4};   // E, F
constexpr uint8_t kByte2High[16] = {
    0, 0, 0, 0, 0, 0, 0, 0,                                          // ASCII (sign mode)
    kCont | kOverlong2 | kOverlong3 | kOverlong4,                    // 1000
    kCont | kOverlong2 | kOverlong3 | kTooLarge,                     // 1001
    kCont | kOverlong2 | kSurrogate | kTooLarge,                     // 1010
    kCont | kOverlong2 | kSurrogate | kTooLarge,                     // 1011
    0, 0, 0, 0};                                                     // leads
constexpr uint8_t kLeadFlags[16] = {
    0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,
    kCont, kCont, kCont | kGeE0, kCont | kGeE0 | kGeF0};

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
constexpr bool allSigns(const uint8_t* t, int from, int to, bool set) {
  return from == to ? true : (((t[from] & 0x80) != 0) == set && allSigns(t, from + 1, to, set));
}
constexpr bool allEqual(const uint8_t* t, int from, int to, uint8_t v) {
  return from == to ? true : (t[from] == v && allEqual(t, from + 1, to, v));
}

constexpr uint32_t kB1H_R0 = highHalfReversed(kByte1High, 0), kB1H_R1 = highHalfReversed(kByte1High, 1);
constexpr uint32_t kB2H_R0 = highHalfReversed(kByte2High, 0), kB2H_R1 = highHalfReversed(kByte2High, 1);
constexpr uint32_t kFlg_R0 = highHalfReversed(kLeadFlags, 0), kFlg_R1 = highHalfReversed(kLeadFlags, 1);
constexpr uint32_t kB1L_L0 = lowHalf(kByte1Low, 0), kB1L_L1 = lowHalf(kByte1Low, 1);
constexpr uint32_t kB1L_R0 = highHalfReversed(kByte1Low, 0), kB1L_R1 = highHalfReversed(kByte1Low, 1);
// prev_side of four zero bytes: byte_1_high of ASCII (0xFF) & byte_1_low[0]
constexpr uint32_t kZeroPrevSide = 0x01010101u * kByte1Low[0];

// What the sign mode produces for ASCII bytes is what the tables say for them.
static_assert(allSigns(kByte1High, 8, 16, true) && allEqual(kByte1High, 0, 8, 0xFF),
              "byte_1_high: sign bits set for 8..F, so ASCII reads 0xFF");
static_assert(allSigns(kByte2High, 8, 16, false) && allEqual(kByte2High, 0, 8, 0),
              "byte_2_high: sign bits clear for 8..F, so ASCII reads 0");
static_assert(allSigns(kLeadFlags, 8, 16, false) && allEqual(kLeadFlags, 0, 8, 0),
              "lead flags: sign bits clear for 8..F, so ASCII reads 0");
static_assert(allSigns(kByte1Low, 0, 16, true),
              "byte_1_low: bit 7 in every entry, so the two half lookups AND to the table");
// Every previous byte carries the continuation bit; only the current side's
// continuations and the expectation decide it.
static_assert((kB1L_L0 & kB1L_L1 & kB1L_R0 & kB1L_R1 & kB1H_R0 & kB1H_R1 & kContBits) == kContBits,
              "the previous side has bit 6 in every entry");

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

// Lookup results for one 32-bit word (four bytes).
struct WordLut {
  uint32_t prev_side;  // byte_1_high[hi] & byte_1_low[lo] of each byte (used as prev1)
  uint32_t cur_side;   // byte_2_high[hi] of each byte
  uint32_t flags;      // lead flags of each byte (0x40: >= 0xC0, 0x20: >= 0xE0, 0x10: >= 0xF0)
};

// Table lookups for one word, given its packed selectors:
//   hi_c     : complemented high nibbles in bits 0..15
//   lo, lo_c : low nibbles and their complements in bits 0..15
__device__ __forceinline__ WordLut lut_from_selectors(uint32_t hi_c, uint32_t lo, uint32_t lo_c) {
  WordLut r;
  r.prev_side = prmt(kB1H_R0, kB1H_R1, hi_c) & prmt(kB1L_L0, kB1L_L1, lo) &
                prmt(kB1L_R0, kB1L_R1, lo_c);
  r.cur_side = prmt(kB2H_R0, kB2H_R1, hi_c);
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
  lc = lut_from_selectors(hi_c, lo, lo_c);
  ld = lut_from_selectors(hi_c >> 16, lo >> 16, lo_c >> 16);
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
  A = lut_from_selectors(hi_c, lo, lo_c);
  B = lut_from_selectors(hi_c >> 16, lo >> 16, lo_c >> 16);
}

// Lookups for byte column 4t..4t+3 of four streams a, b, c, d (natural words),
// as four words W_j = (a_j, b_j, c_j, d_j), j = 0..3: each word holds one
// byte position of the four streams, so the previous bytes of W_j are the
// word before it.  The nibbles of two streams are packed per byte by one
// select each; one byte permute per selector then gathers byte j of both
// packs into the low 16 bits.
__device__ __forceinline__ void lut_quad(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                         WordLut (&W)[4]) {
  const uint32_t lo_mask = 0x0F0F0F0Fu;
  const uint32_t hab = bit_select_not(a >> 4, b, lo_mask);  // byte j: ~(a_j.hi | b_j.hi << 4)
  const uint32_t hcd = bit_select_not(c >> 4, d, lo_mask);
  const uint32_t lab = bit_select(a, b << 4, lo_mask);      // byte j: a_j.lo | b_j.lo << 4
  const uint32_t lcd = bit_select(c, d << 4, lo_mask);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t sel = (uint32_t)(j | ((4 + j) << 4));
    const uint32_t lo = prmt(lab, lcd, sel);
    W[j] = lut_from_selectors(prmt(hab, hcd, sel), lo, ~lo);
  }
}

// The expectation terms of two bytes back and three back, folded per byte:
// bit 6 of byte k of  2 * flags + 4 * prev1_flags  is
// (byte >= 0xE0) XOR (its previous byte >= 0xF0).  (Both terms hold only when
// a lead follows a 4-byte lead directly, an error that the continuation
// check catches at that lead, so XOR in place of OR never hides an error.)
// Carries stay below bit 7 of the byte or spill into bits 0..1 of the next
// byte, outside bit 6.  Integer multiplies: the FMA pipe, not the ALU pipe.
__device__ __forceinline__ uint32_t back23(uint32_t flags, uint32_t prev1_flags) {
  return flags * 2u + prev1_flags * 4u;
}

// Error byte of each position of a word, given the word's lookups, its
// previous bytes' lookups aligned to it (prev1 = x, flags of prev1 = g) and
// back23 of the bytes two back (h2).  Non-zero iff the position is an error.
__device__ __forceinline__ uint32_t position_errors(uint32_t x, uint32_t cur_side, uint32_t g,
                                                    uint32_t h2) {
  const uint32_t expect = (g | h2) & kContBits;
  return (x & cur_side) ^ expect;
}

// Error bytes of a natural-order word `cur` after the four bytes whose
// prev_side, flags and back23 are p, f and h (bytes 1..3 used; h's byte 1 is
// not needed).
__device__ __forceinline__ uint32_t word_error_after(uint32_t p, uint32_t f, uint32_t h,
                                                     const WordLut& cur) {
  const uint32_t x = __funnelshift_l(p, cur.prev_side, 8);
  const uint32_t g = __funnelshift_l(f, cur.flags, 8);
  const uint32_t hc = back23(cur.flags, g);
  return position_errors(x, cur.cur_side, g, __funnelshift_l(h, hc, 16));
}

// back23 of a natural-order word on its own: exact in bytes 1..3.
__device__ __forceinline__ uint32_t back23_word(const WordLut& w) {
  return back23(w.flags, w.flags << 8);
}

// Error bytes of the four positions of `cur` (natural order) after `prev`.
__device__ __forceinline__ uint32_t word_error(const WordLut& prev, const WordLut& cur) {
  return word_error_after(prev.prev_side, prev.flags, back23_word(prev), cur);
}

// Lookups of four zero bytes (the ASCII padding before and after a stream).
__device__ __forceinline__ WordLut ascii_lut() {
  WordLut r;
  r.prev_side = kZeroPrevSide;
  r.cur_side = 0;
  r.flags = 0;
  return r;
}

}  // namespace utf8gpu

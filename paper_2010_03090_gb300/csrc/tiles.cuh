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

// What lane 0 of a row group needs from the row group before it: lookups of
// the last word of lane 31 (the last bytes of every row).
//  * Row pairs: interleaved word W_7 (the last four bytes of both rows): its
//    prev_side, flags and back23 in p, f and hb; the second-stream bytes (1
//    and 3) are used.
//  * Row quads: word W_15 (byte 15 of the four rows): its prev_side and flags
//    in p and f, back23 of W_14 and W_15 in ha and hb; byte 3 (the quad's last
//    row) is used.
struct Carry {
  uint32_t p;
  uint32_t f;
  uint32_t ha;
  uint32_t hb;
};

// Rows are classified four at a time when the tile height allows it (see
// check_tile); a kernel may ask for row pairs instead.
template <int ROWS>
constexpr bool kQuadRows = ROWS % 4 == 0;

__device__ __forceinline__ Carry ascii_carry() {
  const WordLut a = ascii_lut();
  return Carry{a.prev_side, a.flags, 0u, 0u};
}

// Carry for a stream whose previous four bytes (natural order) are `halo`.
template <bool QUADS>
__device__ __forceinline__ Carry halo_carry(uint32_t halo) {
  const WordLut h = lut_word(halo);
  const uint32_t b = back23_word(h);  // byte k: back23 of halo byte k (k = 2, 3 exact)
  if constexpr (QUADS) return Carry{h.prev_side, h.flags, b << 8, b};
  return Carry{prmt(h.prev_side, 0, 0x3020), prmt(h.flags, 0, 0x3020), 0u, prmt(b, 0, 0x3020)};
}

// Error bytes of the first four positions of a tile's row 0 (natural order,
// word w) after the carry: the check an all-ASCII tile still makes.
template <bool QUADS>
__device__ __forceinline__ uint32_t word_error_after_carry(const Carry& c, uint32_t w) {
  if constexpr (QUADS) {
    // byte 3 of each carry word is the last byte before the tile
    return word_error_after(c.p, c.f, prmt(c.ha, c.hb, 0x7300), lut_word(w));
  }
  // the carry's stream-1 bytes 1 and 3 are the last two bytes before the tile
  return word_error_after(prmt(c.p, 0, 0x3144), prmt(c.f, 0, 0x3144), prmt(c.hb, 0, 0x3144),
                          lut_word(w));
}

template <int ROWS>
struct TileGeom {
  static constexpr uint64_t kGranules = (uint64_t)kLanes * ROWS;
  static constexpr uint64_t kBytes = kGranules * 16;
};

// Tile t with bounds checks (first and last tiles of a stream).
template <int ROWS>
__device__ __forceinline__ void load_tile_checked(const Span& s, uint64_t t, int lane,
                                                  uint4 (&d)[ROWS]) {
  const uint64_t g0 = t * TileGeom<ROWS>::kGranules;
#pragma unroll
  for (int r = 0; r < ROWS; ++r) d[r] = load_granule(s, g0 + r * kLanes + lane);
}

// Tile wholly inside the data: lane_ptr = abase + t * tile bytes + lane * 16.
template <int ROWS>
__device__ __forceinline__ void load_tile_interior(const uint8_t* lane_ptr, uint4 (&d)[ROWS]) {
#pragma unroll
  for (int r = 0; r < ROWS; ++r) d[r] = ld_stream(lane_ptr + r * kLanes * 16);
}

// Tile t, unchecked when it is interior (in0 <= t < in1), checked otherwise.
template <int ROWS>
__device__ __forceinline__ void load_tile(const Span& s, uint64_t t, uint64_t in0, uint64_t in1,
                                          int lane, const uint8_t* lane_ptr, uint4 (&d)[ROWS]) {
  if (t >= in0 && t < in1) load_tile_interior<ROWS>(lane_ptr, d);
  else load_tile_checked<ROWS>(s, t, lane, d);
}

// Interior tiles of a stream: [first, last) (every granule inside [off, off + n)).
template <int ROWS>
__device__ __forceinline__ void interior_tiles(const Span& s, uint64_t& first, uint64_t& last) {
  constexpr uint64_t tb = TileGeom<ROWS>::kBytes;
  first = (s.off + tb - 1) / tb;
  last = (s.off + s.n) / tb;
}

// Checks one loaded tile.  e holds ROWS * 4 error words per lane, e[i / 8][i % 8]
// for word i; a position is an error iff its byte is non-zero
// (interleaved_position gives each byte's position).
//  * QUADS (the default where ROWS is a multiple of 4): rows 4q .. 4q+3 are
//    processed together as four streams, word i = 16q + k being W_k = (byte k
//    of row 4q, of row 4q+1, of row 4q+2, of row 4q+3) of this lane's granules
//    (see lut_quad): byte j's previous bytes are byte j of W_{k-1}, W_{k-2},
//    W_{k-3}.
//  * Row pairs: rows 2p and 2p+1 are processed as two interleaved streams,
//    word i = 8p + m being W_m = (row 2p byte 2m, row 2p+1 byte 2m, row 2p
//    byte 2m+1, row 2p+1 byte 2m+1) (see lut_interleaved); the previous bytes
//    are a 16-bit funnel shift away.
// `carry` describes the bytes before the tile (lane 0) and is updated.
//
// The all-ASCII test first votes on the tile's first row (512 bytes) alone:
// on text with non-ASCII characters that row almost always holds one, and the
// tile goes straight to the classification without OR-ing its other rows;
// only a tile whose first row is ASCII pays for the full test.
template <int ROWS, bool QUADS = kQuadRows<ROWS>>
__device__ __forceinline__ void check_tile(const uint4 (&d)[ROWS], Carry& carry, int lane,
                                           uint32_t merge_sel, uint32_t (&e)[ROWS / 2][8]) {
  static_assert(QUADS ? ROWS % 4 == 0 : ROWS % 2 == 0, "whole row groups");
  const int left = (lane + kLanes - 1) & (kLanes - 1);
  const uint32_t sample = d[0].x | d[0].y | d[0].z | d[0].w;
  bool ascii = false;
  if (!__any_sync(kFull, sample & 0x80808080u)) {
    uint32_t high = sample;
#pragma unroll
    for (int r = 1; r < ROWS; ++r) high |= d[r].x | d[r].y | d[r].z | d[r].w;
    ascii = !__any_sync(kFull, high & 0x80808080u);
  }
  if (ascii) {
    // All-ASCII tile (Section 6.4): no classification, but the bytes before
    // the tile must not end inside a character.
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) e[p][m] = 0;
    if (lane == 0) {
      const uint32_t first = word_error_after_carry<QUADS>(carry, d[0].x);
      if constexpr (QUADS) {
        // positions 0..3 of row 0: byte 0 of W_0 .. W_3
        e[0][0] = first & 0xFFu;
        e[0][1] = (first >> 8) & 0xFFu;
        e[0][2] = (first >> 16) & 0xFFu;
        e[0][3] = first >> 24;
      } else {
        e[0][0] = prmt(first, 0, 0x4140);  // positions 0, 1 of row 0
        e[0][1] = prmt(first, 0, 0x4342);  // positions 2, 3 of row 0
      }
    }
    carry = ascii_carry();
    return;
  }
  if constexpr (QUADS) {
#pragma unroll
    for (int q = 0; q < ROWS / 4; ++q) {
      const uint4 a = d[4 * q], b = d[4 * q + 1], c = d[4 * q + 2], dd = d[4 * q + 3];
      WordLut W[16];
      lut_quad(a.x, b.x, c.x, dd.x, *reinterpret_cast<WordLut(*)[4]>(&W[0]));
      lut_quad(a.y, b.y, c.y, dd.y, *reinterpret_cast<WordLut(*)[4]>(&W[4]));
      lut_quad(a.z, b.z, c.z, dd.z, *reinterpret_cast<WordLut(*)[4]>(&W[8]));
      lut_quad(a.w, b.w, c.w, dd.w, *reinterpret_cast<WordLut(*)[4]>(&W[12]));
      uint32_t h[16];
#pragma unroll
      for (int k = 1; k < 16; ++k) h[k] = back23(W[k].flags, W[k - 1].flags);
      // left neighbour's W_15; lane 0 takes row 0 from the carry (the row
      // before the quad) and rows 1..3 from rows 0..2 of lane 31
      const uint32_t p15 = __shfl_sync(kFull, W[15].prev_side, left);
      const uint32_t f15 = __shfl_sync(kFull, W[15].flags, left);
      const uint32_t h14 = __shfl_sync(kFull, h[14], left);
      const uint32_t h15 = __shfl_sync(kFull, h[15], left);
      const uint32_t lp = prmt(carry.p, p15, merge_sel);
      const uint32_t lf = prmt(carry.f, f15, merge_sel);
      const uint32_t lh14 = prmt(carry.ha, h14, merge_sel);
      const uint32_t lh15 = prmt(carry.hb, h15, merge_sel);
      carry = Carry{p15, f15, h14, h15};
      h[0] = back23(W[0].flags, lf);
      uint32_t* eq = &e[2 * q][0];
      eq[0] = position_errors(lp, W[0].cur_side, lf, lh14);
      eq[1] = position_errors(W[0].prev_side, W[1].cur_side, W[0].flags, lh15);
#pragma unroll
      for (int k = 2; k < 16; ++k)
        eq[k] = position_errors(W[k - 1].prev_side, W[k].cur_side, W[k - 1].flags, h[k - 2]);
    }
  } else {
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p) {
      const uint4 c = d[2 * p], n = d[2 * p + 1];
      WordLut W[8];
      lut_interleaved(c.x, n.x, W[0], W[1]);
      lut_interleaved(c.y, n.y, W[2], W[3]);
      lut_interleaved(c.z, n.z, W[4], W[5]);
      lut_interleaved(c.w, n.w, W[6], W[7]);
      // flags of each word's previous bytes (prev1) and back23 of each word
      uint32_t g[8], h[8];
#pragma unroll
      for (int m = 1; m < 8; ++m) {
        g[m] = __funnelshift_l(W[m - 1].flags, W[m].flags, 16);
        h[m] = back23(W[m].flags, g[m]);
      }
      // left neighbour's W_7; lane 0 takes its first stream from the carry
      // (the row before) and its second stream from lane 31 of the first row
      const uint32_t x7 = __shfl_sync(kFull, W[7].prev_side, left);
      const uint32_t f7 = __shfl_sync(kFull, W[7].flags, left);
      const uint32_t h7 = __shfl_sync(kFull, h[7], left);
      const uint32_t lx = prmt(carry.p, x7, merge_sel);
      const uint32_t lf = prmt(carry.f, f7, merge_sel);
      const uint32_t lh = prmt(carry.hb, h7, merge_sel);
      carry = Carry{x7, f7, 0u, h7};
      g[0] = __funnelshift_l(lf, W[0].flags, 16);
      h[0] = back23(W[0].flags, g[0]);
      e[p][0] = position_errors(__funnelshift_l(lx, W[0].prev_side, 16), W[0].cur_side, g[0], lh);
#pragma unroll
      for (int m = 1; m < 8; ++m)
        e[p][m] = position_errors(__funnelshift_l(W[m - 1].prev_side, W[m].prev_side, 16),
                                  W[m].cur_side, g[m], h[m - 1]);
    }
  }
}

// Virtual position (relative to the tile start) of byte b of error word
// e[p][m] in lane `lane` (see check_tile).
template <int ROWS, bool QUADS = kQuadRows<ROWS>>
__device__ __forceinline__ uint32_t interleaved_position(int p, int m, int b, int lane) {
  if constexpr (QUADS) {
    const int i = p * 8 + m;
    const int row = 4 * (i >> 4) + b;
    return (uint32_t)(row * kLanes + lane) * 16u + (uint32_t)(i & 15);
  }
  const int row = 2 * p + (b & 1);
  return (uint32_t)(row * kLanes + lane) * 16u + (uint32_t)(2 * m + (b >> 1));
}

// Selector merging the carry into lane 0's left neighbour (see check_tile).
template <bool QUADS>
__device__ __forceinline__ uint32_t carry_merge_selector(int lane) {
  if constexpr (QUADS) return lane == 0 ? 0x6543u : 0x7654u;
  return lane == 0 ? 0x6341u : 0x7654u;
}

// A result byte that several warps of one grid may clear while the others
// still run: GPU-scope relaxed accesses, so that a store by one warp is seen by
// the loads of the others (through L2, never a stale L1 line).  The byte is 1
// before the launch and only ever cleared, so a warp that reads 0 knows the
// answer is final.
__device__ __forceinline__ uint32_t load_result(const uint8_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void clear_result(uint8_t* p) {
  asm volatile("st.relaxed.gpu.global.u8 [%0], %1;" ::"l"(p), "r"(0u));
}

// One warp's run of tiles [t_begin, t_begin + cnt) of a stream, counted from
// t_begin in 32 bits (a run is far below 2^32 tiles): the run's interior
// tiles are [i0, i0 + i_len).  With 32-bit counters the loop's own
// bookkeeping takes fewer instructions from the ALU pipe that bounds the
// classification.
struct RunTiles {
  uint32_t cnt;
  uint32_t i0;
  uint32_t i_len;
};

template <int ROWS>
__device__ __forceinline__ RunTiles run_tiles(const Span& s, uint64_t t_begin, uint64_t t_end) {
  uint64_t in0, in1;
  interior_tiles<ROWS>(s, in0, in1);
  RunTiles r;
  r.cnt = t_end > t_begin ? (uint32_t)(t_end - t_begin) : 0u;
  const uint64_t c0 = in0 > t_begin ? in0 - t_begin : 0;
  const uint64_t c1 = in1 > t_begin ? in1 - t_begin : 0;
  r.i0 = (uint32_t)(c0 < r.cnt ? c0 : r.cnt);
  const uint32_t i1 = (uint32_t)(c1 < r.cnt ? c1 : r.cnt);
  r.i_len = i1 > r.i0 ? i1 - r.i0 : 0u;
  return r;
}

// Tile t_begin + k of a run; p = abase + (t_begin + k) * tile bytes + lane * 16.
template <int ROWS>
__device__ __forceinline__ void load_run_tile(const Span& s, const RunTiles& r, uint64_t t_begin,
                                              uint32_t k, int lane, const uint8_t* p,
                                              uint4 (&d)[ROWS]) {
  if (k - r.i0 < r.i_len) load_tile_interior<ROWS>(p, d);
  else load_tile_checked<ROWS>(s, t_begin + k, lane, d);
}

// Bytes a polling warp checks between two looks at a result.
constexpr uint32_t kPollBytes = 16 << 10;

// Checks tiles [t_begin, t_end) of a stream (t_begin <= t_end) with one warp;
// returns a non-zero value in some lane iff an error lies in those tiles.
// The next tile's loads are issued before the current tile is classified, so
// their latency overlaps the ALU-bound classification.  Tile counts relative
// to t_begin fit 32 bits (a run is far below 2^32 tiles); the interior tiles
// of the run are [i0, i0 + i_len).  The run is set up here as in run_tiles,
// written out: through run_tiles and load_run_tile this loop compiled 0.8%
// slower.
template <int ROWS, bool QUADS = kQuadRows<ROWS>>
__device__ __forceinline__ uint32_t warp_check_tiles(const Span& s, uint64_t t_begin,
                                                     uint64_t t_end) {
  constexpr uint64_t tb = TileGeom<ROWS>::kBytes;
  const int lane = threadIdx.x & (kLanes - 1);
  uint32_t err = 0;
  const uint32_t merge_sel = carry_merge_selector<QUADS>(lane);
  Carry carry = ascii_carry();  // zeros before the stream
  if (t_begin < t_end && t_begin > 0) carry = halo_carry<QUADS>(load_word(s, t_begin * tb - 4));
  uint64_t in0, in1;
  interior_tiles<ROWS>(s, in0, in1);
  const uint8_t* lane_ptr = s.abase + t_begin * tb + lane * 16;
  const uint32_t cnt = (uint32_t)(t_end - t_begin);
  const uint64_t c0 = in0 > t_begin ? in0 - t_begin : 0;
  const uint64_t c1 = in1 > t_begin ? in1 - t_begin : 0;
  const uint32_t i0 = (uint32_t)(c0 < cnt ? c0 : cnt);
  const uint32_t i1 = (uint32_t)(c1 < cnt ? c1 : cnt);
  const uint32_t i_len = i1 > i0 ? i1 - i0 : 0;
  const auto load_rel = [&](uint32_t k, const uint8_t* p, uint4 (&d)[ROWS]) {
    if (k - i0 < i_len) load_tile_interior<ROWS>(p, d);
    else load_tile_checked<ROWS>(s, t_begin + k, lane, d);
  };
  uint4 next[ROWS];
  if (cnt > 0) load_rel(0, lane_ptr, next);
  for (uint32_t k = 0; k < cnt; ++k, lane_ptr += tb) {
    uint4 d[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) d[r] = next[r];
    if (k + 1 < cnt) load_rel(k + 1, lane_ptr + tb, next);
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS, QUADS>(d, carry, lane, merge_sel, e);
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) err |= e[p][m];
  }
  return err;
}

// warp_check_tiles that stops early once the stream's answer is known to be
// "invalid".  Every kPollBytes the warp votes on the errors it has found so
// far and looks at the result byte it loaded kPollBytes earlier (so the
// load's latency hides behind the classification), and leaves if either
// shows an error; errors in the tiles it skips cannot change the answer.
// The split loop costs about 2% of the classification rate on valid text
// (the single loop above schedules better), so polling is the caller's choice.
template <int ROWS, bool QUADS = kQuadRows<ROWS>>
__device__ __forceinline__ uint32_t warp_check_tiles_polling(const Span& s, uint64_t t_begin,
                                                             uint64_t t_end,
                                                             const uint8_t* result) {
  constexpr uint64_t tb = TileGeom<ROWS>::kBytes;
  constexpr uint32_t poll_tiles = kPollBytes / (uint32_t)tb;
  static_assert(poll_tiles >= 1, "a poll falls after whole tiles");
  const int lane = threadIdx.x & (kLanes - 1);
  uint32_t err = 0;
  const uint32_t merge_sel = carry_merge_selector<QUADS>(lane);
  Carry carry = ascii_carry();  // zeros before the stream
  if (t_begin < t_end && t_begin > 0) carry = halo_carry<QUADS>(load_word(s, t_begin * tb - 4));
  const RunTiles run = run_tiles<ROWS>(s, t_begin, t_end);
  const uint8_t* lane_ptr = s.abase + t_begin * tb + lane * 16;
  const bool poll = poll_tiles < run.cnt;
  uint32_t seen = poll ? load_result(result) : 1u;
  uint4 next[ROWS];
  if (run.cnt > 0) load_run_tile<ROWS>(s, run, t_begin, 0, lane, lane_ptr, next);
  uint32_t k = 0;
  while (k < run.cnt) {
    const uint32_t k_look = poll && run.cnt - k > poll_tiles ? k + poll_tiles : run.cnt;
    for (; k < k_look; ++k, lane_ptr += tb) {
      uint4 d[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) d[r] = next[r];
      if (k + 1 < run.cnt)
        load_run_tile<ROWS>(s, run, t_begin, k + 1, lane, lane_ptr + tb, next);
      uint32_t e[ROWS / 2][8];
      check_tile<ROWS, QUADS>(d, carry, lane, merge_sel, e);
#pragma unroll
      for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
        for (int m = 0; m < 8; ++m) err |= e[p][m];
    }
    if (k < run.cnt) {  // only when polling
      if (__any_sync(kFull, err != 0 || seen == 0)) break;
      seen = load_result(result);
    }
  }
  return err;
}

// ---------------------------------------------------------------------------
// Staged form of warp_check_tiles: the coming tiles are copied into shared
// memory with cp.async, kStages - 1 tiles ahead of the one being classified,
// so no register holds a tile in flight (the register form keeps the next
// tile in 32 registers, one tile ahead).  The deeper lead and the freed
// registers measured 4% faster on non-ASCII text at 8 rows.
//
// `ring` is this warp's kStages slots of ROWS * 32 granules in shared memory.
// Each lane copies, and later reads back, only its own granules of a slot,
// so the lanes need no barrier: cp.async.wait_group makes a lane wait for its
// own copies.  A slot is refilled only after the lane has classified the tile
// it held (every loaded word feeds the classification before the refill is
// issued).  The first and last tiles of a stream take the checked loads and
// are stored to the slot directly.
// ---------------------------------------------------------------------------
constexpr int kStages = 3;

// Shared memory of the rings of one CTA of `threads` threads.
template <int ROWS>
constexpr int staged_smem_bytes(int threads) {
  return (threads / kLanes) * kStages * ROWS * kLanes * 16;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One warp's run of tiles through its ring: start() issues the first
// kStages - 1 tiles; next(k, d) issues tile k + kStages - 1, waits for tile k
// (the lane's own copies) and loads the lane's granules of it into d;
// finish() waits for every copy still in flight (before a warp leaves early
// or ends).  Tiles are taken in order, k = 0, 1, ...
template <int ROWS>
struct StagedRun {
  static constexpr int kSlot = ROWS * kLanes;  // granules per slot
  const Span& s;
  RunTiles run;
  uint64_t t_begin;
  const uint8_t* lane_ptr;  // abase + t_begin * tile bytes + lane * 16
  uint4* ring;
  int lane;
  int rd = 0, wr = kStages - 1;

  __device__ __forceinline__ StagedRun(const Span& s_, uint64_t t_begin_, uint64_t t_end,
                                       uint4* ring_, int lane_)
      : s(s_), run(run_tiles<ROWS>(s_, t_begin_, t_end)), t_begin(t_begin_),
        lane_ptr(s_.abase + t_begin_ * TileGeom<ROWS>::kBytes + lane_ * 16), ring(ring_),
        lane(lane_) {}

  // tile t_begin + k into a slot: cp.async when interior, checked loads else
  __device__ __forceinline__ void issue(uint32_t k, uint4* slot) const {
    if (k - run.i0 < run.i_len) {
      const uint8_t* p = lane_ptr + (uint64_t)k * TileGeom<ROWS>::kBytes;
#pragma unroll
      for (int r = 0; r < ROWS; ++r) cp_async16(&slot[r * kLanes + lane], p + r * kLanes * 16);
    } else {
      const uint64_t g0 = (t_begin + k) * TileGeom<ROWS>::kGranules;
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
        slot[r * kLanes + lane] = load_granule(s, g0 + r * kLanes + lane);
    }
  }
  __device__ __forceinline__ void start() const {
#pragma unroll
    for (int j = 0; j < kStages - 1; ++j) {
      if ((uint32_t)j < run.cnt) issue((uint32_t)j, ring + j * kSlot);
      cp_async_commit();
    }
  }
  __device__ __forceinline__ void next(uint32_t k, uint4 (&d)[ROWS]) {
    if (k + kStages - 1 < run.cnt) issue(k + kStages - 1, ring + wr * kSlot);
    cp_async_commit();  // one group per tile, empty or not
    cp_async_wait<kStages - 1>();  // tile k's group is complete
    const uint4* slot = ring + rd * kSlot;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) d[r] = slot[r * kLanes + lane];
    rd = rd + 1 == kStages ? 0 : rd + 1;
    wr = wr + 1 == kStages ? 0 : wr + 1;
  }
  __device__ __forceinline__ void finish() const { cp_async_wait<0>(); }
};

template <int ROWS, bool QUADS = kQuadRows<ROWS>>
__device__ __forceinline__ uint32_t warp_check_tiles_staged(const Span& s, uint64_t t_begin,
                                                            uint64_t t_end, uint4* ring) {
  constexpr uint64_t tb = TileGeom<ROWS>::kBytes;
  const int lane = threadIdx.x & (kLanes - 1);
  uint32_t err = 0;
  const uint32_t merge_sel = carry_merge_selector<QUADS>(lane);
  Carry carry = ascii_carry();  // zeros before the stream
  if (t_begin < t_end && t_begin > 0) carry = halo_carry<QUADS>(load_word(s, t_begin * tb - 4));
  StagedRun<ROWS> st(s, t_begin, t_end, ring, lane);
  st.start();
  for (uint32_t k = 0; k < st.run.cnt; ++k) {
    uint4 d[ROWS];
    st.next(k, d);
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS, QUADS>(d, carry, lane, merge_sel, e);
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) err |= e[p][m];
  }
  st.finish();
  return err;
}

// warp_check_tiles_polling through the ring: every kPollBytes the warp votes
// on the errors it has found and looks at the result byte it loaded
// kPollBytes earlier, and leaves (after its copies in flight) once either
// shows an error.
template <int ROWS, bool QUADS = kQuadRows<ROWS>>
__device__ __forceinline__ uint32_t warp_check_tiles_staged_polling(const Span& s, uint64_t t_begin,
                                                                    uint64_t t_end, uint4* ring,
                                                                    const uint8_t* result) {
  constexpr uint64_t tb = TileGeom<ROWS>::kBytes;
  constexpr uint32_t poll_tiles = kPollBytes / (uint32_t)tb;
  static_assert(poll_tiles >= 1, "a poll falls after whole tiles");
  const int lane = threadIdx.x & (kLanes - 1);
  uint32_t err = 0;
  const uint32_t merge_sel = carry_merge_selector<QUADS>(lane);
  Carry carry = ascii_carry();  // zeros before the stream
  if (t_begin < t_end && t_begin > 0) carry = halo_carry<QUADS>(load_word(s, t_begin * tb - 4));
  StagedRun<ROWS> st(s, t_begin, t_end, ring, lane);
  const bool poll = poll_tiles < st.run.cnt;
  uint32_t seen = poll ? load_result(result) : 1u;
  st.start();
  uint32_t to_look = poll_tiles;
  for (uint32_t k = 0; k < st.run.cnt; ++k) {
    uint4 d[ROWS];
    st.next(k, d);
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS, QUADS>(d, carry, lane, merge_sel, e);
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) err |= e[p][m];
    if (poll && --to_look == 0 && k + 1 < st.run.cnt) {
      to_look = poll_tiles;
      if (__any_sync(kFull, err != 0 || seen == 0)) break;
      seen = load_result(result);
    }
  }
  st.finish();
  return err;
}

}  // namespace utf8gpu

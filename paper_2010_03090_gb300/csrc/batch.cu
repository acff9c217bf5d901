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

// The 8 bytes [x, x + 8) of `data` (absolute offsets) as two words, bytes
// outside [lo, hi) zero.  Only the aligned 4-byte words holding a byte of
// [lo, hi) are read; [lo, hi) lies inside the batch region, so those words lie
// in granules the stream reads anyway.
__device__ __forceinline__ void gather8(const uint8_t* data, int64_t x, int64_t lo, int64_t hi,
                                        uint32_t& w_lo, uint32_t& w_hi) {
  const int64_t a = lo > x ? lo : x;
  const int64_t b = hi < x + 8 ? hi : x + 8;
  w_lo = w_hi = 0u;
  if (a >= b) return;
  const uintptr_t px = reinterpret_cast<uintptr_t>(data + x);
  const int sh = (int)(px & 3u);
  const uint32_t* base = reinterpret_cast<const uint32_t*>(px - (uintptr_t)sh);
  const int ka = (int)(a - x), kb = (int)(b - x);  // wanted bytes [ka, kb) of the 8, 0 <= ka < kb <= 8
  uint32_t u[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int ws = 4 * k - sh;  // word k holds bytes [ws, ws + 4) of the 8
    u[k] = (ws < kb && ws + 4 > ka) ? __ldg(base + k) : 0u;
  }
  const uint32_t s8 = 8u * (uint32_t)sh;
  w_lo = __funnelshift_r(u[0], u[1], s8) & keep_bytes(ka, kb);
  w_hi = __funnelshift_r(u[1], u[2], s8) & keep_bytes(ka - 4, kb - 4);
}

// First j in [0, hi) with offsets[j] >= target (hi if none), for two targets
// at once; whole warp (search.cuh gives the narrowing step).  Each round every
// lane probes both ranges, so the two chains of dependent loads overlap: a
// warp's start waits for the rounds of one search, not of two.
__device__ void warp_lower_bound2(const int64_t* offsets, int64_t hi, int64_t target_a,
                                  int64_t target_b, int64_t& res_a, int64_t& res_b) {
  const int lane = threadIdx.x & (kLanes - 1);
  int64_t lo_a = 0, hi_a = hi, lo_b = 0, hi_b = hi;
  while (hi_a - lo_a > kLanes || hi_b - lo_b > kLanes) {
    const bool open_a = hi_a - lo_a > kLanes, open_b = hi_b - lo_b > kLanes;
    const int64_t step_a = lb_step(lo_a, hi_a), step_b = lb_step(lo_b, hi_b);
    const int64_t ja = lo_a + lane * step_a, jb = lo_b + lane * step_b;
    const bool ge_a = open_a && ja < hi_a ? offsets[ja] >= target_a : true;
    const bool ge_b = open_b && jb < hi_b ? offsets[jb] >= target_b : true;
    const uint32_t mask_a = __ballot_sync(kFull, ge_a);
    const uint32_t mask_b = __ballot_sync(kFull, ge_b);
    if (open_a) {
      const LbRange r = lb_narrow(lo_a, hi_a, step_a, mask_a);
      lo_a = r.lo;
      hi_a = r.hi;
    }
    if (open_b) {
      const LbRange r = lb_narrow(lo_b, hi_b, step_b, mask_b);
      lo_b = r.lo;
      hi_b = r.hi;
    }
  }
  const int64_t ja = lo_a + lane, jb = lo_b + lane;
  const bool ge_a = ja < hi_a ? offsets[ja] >= target_a : true;
  const bool ge_b = jb < hi_b ? offsets[jb] >= target_b : true;
  const uint32_t mask_a = __ballot_sync(kFull, ge_a);
  const uint32_t mask_b = __ballot_sync(kFull, ge_b);
  res_a = lb_final(lo_a, hi_a, mask_a);
  res_b = lb_final(lo_b, hi_b, mask_b);
}

// The batch pass classifies row quads where the tile height allows
// (tiles.cuh).  Its tiles come through a ring of kStages slots per warp in
// shared memory, filled by cp.async two tiles ahead: no register holds a tile
// in flight, which leaves room for the quads' state beside the boundary and
// charging state (with register loads quads took 169 registers, one CTA per
// SM, and ran 2.6% slower than row pairs).
template <int ROWS>
constexpr bool kBatchQuads = kQuadRows<ROWS>;
// A slot: the 8 bytes before its tile (header bytes 8..15), then the tile,
// in 32-bit words.
template <int ROWS>
constexpr int kBatchSlotWords = 4 + ROWS * 32 * 4;
// Dynamic shared memory of one CTA's rings.
template <int ROWS>
constexpr int batch_smem_bytes() {
  return (kBlockThreads / 32) * kStages * kBatchSlotWords<ROWS> * 4;
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
__device__ __forceinline__ void batch_body(const uint8_t* __restrict__ data,
                                           const int64_t* __restrict__ offsets, int64_t count,
                                           uint8_t* __restrict__ out_valid,
                                           utf8_error_info* out_err) {
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

  // Per warp: the 8 bytes before the current tile (bytes 8..15), then the
  // tile itself (from byte 16), staged so that boundary windows are taken
  // from it instead of being read again from memory.  A tile with errors
  // reuses the tile part for its error words once its windows are taken.
  constexpr int kSlotWords = kBatchSlotWords<ROWS>;
  extern __shared__ __align__(16) uint32_t batch_rings[];
  uint32_t* const ring = batch_rings + (threadIdx.x / kLanes) * kStages * kSlotWords;
  uint32_t* stage = ring;
  uint32_t* err_words = stage + 4;
  // Tiles are counted from t0 in 32 bits (a warp's run is far below 2^32
  // tiles); [r_in0, r_in1) are its tiles wholly inside the region.
  const uint32_t n_tiles = (uint32_t)(t1 - t0);
  uint64_t in0, in1;
  interior_tiles<ROWS>(region, in0, in1);
  const uint32_t r_in0 = (uint32_t)(in0 <= t0 ? 0 : (in0 - t0 < n_tiles ? in0 - t0 : n_tiles));
  const uint32_t r_in1 = (uint32_t)(in1 <= t0 ? 0 : (in1 - t0 < n_tiles ? in1 - t0 : n_tiles));
  const uint8_t* lane_ptr = region.abase + t0 * kTileBytes + lane * 16;
  // the first tiles' copies go out before the boundary search
  // tile t0 + k into its slot (data after the 16-byte header): cp.async when
  // the tile lies inside the region, checked loads stored directly else
  const auto issue = [&](uint32_t k) {
    uint4* slot = reinterpret_cast<uint4*>(ring + (k % kStages) * kSlotWords + 4);
    if (k >= r_in0 && k < r_in1) {
      const uint8_t* p = lane_ptr + (uint64_t)k * kTileBytes;
#pragma unroll
      for (int r = 0; r < ROWS; ++r) cp_async16(&slot[r * kLanes + lane], p + r * kLanes * 16);
    } else {
      uint4 c[ROWS];
      load_tile_checked<ROWS>(region, t0 + k, lane, c);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) slot[r * kLanes + lane] = c[r];
    }
  };
  issue(0);
  cp_async_commit();
  if (n_tiles > 1) issue(1);
  cp_async_commit();
  int rd = 0;
  // absolute offset of virtual position 0 of the region
  const int64_t vbase = o_first - (int64_t)region.off;
  const int64_t range_lo = vbase + (int64_t)(t0 * kTileBytes);
  const int64_t range_hi = vbase + (int64_t)(t1 * kTileBytes);
  // boundaries of this warp: offsets[j] in [range_lo, range_hi), j in [b0, b1)
  int64_t b0, b1;
  warp_lower_bound2(offsets, count + 1, range_lo, range_hi, b0, b1);
  // strings that can hold a position of this warp: b0 - 1 .. b1 - 1
  const int64_t own_hi = b1 < count ? b1 : count;

  static_assert(ROWS / 2 * 8 * kLanes == ROWS * kLanes * 4, "error words fit the tile part");

  const uint32_t merge_sel = carry_merge_selector<kBatchQuads<ROWS>>(lane);
  Carry carry = ascii_carry();
  const uint32_t halo = t0 > 0 ? load_word(region, t0 * kTileBytes - 4) : 0u;
  if (t0 > 0) carry = halo_carry<kBatchQuads<ROWS>>(halo);
  if (lane == 0) {
    stage[2] = t0 > 0 ? load_word(region, t0 * kTileBytes - 8) : 0u;
    stage[3] = halo;
  }

  // Boundary groups of up to 32, [next_group, group_last]; lane k holds
  // g_off = offsets[next_group + k] (INT64_MAX past the group) and every lane
  // holds prev_off = offsets[next_group - 1].  A group is checked on the tile
  // holding its last boundary (tile `due`, counted from t0) or on the warp's
  // last tile, so its bytes are recent in L2.
  // The offsets of the group after the open one are loaded when it opens
  // (g_nxt), so opening a group waits for no load.
  int64_t next_group = b0;
  int64_t group_last = -1;
  int64_t g_off = INT64_MAX;
  // The window [o_j - 4, o_j + 4) of this lane's boundary, taken from the
  // staged tile holding its last byte; `win_global` when that tile's staged
  // bytes were already replaced (then it is read from memory at the check).
  uint32_t win_lo = 0, win_hi = 0;
  bool win_global = false;
  int64_t prev_off = b0 > 0 ? offsets[b0 - 1] : INT64_MIN;
  uint32_t due = 0xFFFFFFFFu;
  auto group_offsets = [&](int64_t first) -> int64_t {
    const int64_t last = (first + kLanes < b1 ? first + kLanes : b1) - 1;
    return first + lane <= last ? offsets[first + lane] : INT64_MAX;
  };
  int64_t g_nxt = b0 < b1 ? group_offsets(b0) : INT64_MAX;
  auto open_group = [&]() {
    if (next_group < b1) {
      group_last = (next_group + kLanes < b1 ? next_group + kLanes : b1) - 1;
      g_off = g_nxt;
      const int64_t last_off = __shfl_sync(kFull, g_off, (int)(group_last - next_group));
      // checked on the tile holding the last byte of its last window
      due = (uint32_t)(((uint64_t)(last_off + 3 - vbase) / kTileBytes) - t0);
      win_global = false;
      g_nxt = group_last + 1 < b1 ? group_offsets(group_last + 1) : INT64_MAX;
    } else {
      g_off = INT64_MAX;
      due = 0xFFFFFFFFu;
    }
  };
  open_group();

  // Takes the windows that end in the staged tile starting at tile_lo.
  auto take_windows = [&](int64_t tile_lo, bool staged) {
    const int64_t end = g_off + 3 - tile_lo;  // last window byte, tile-relative
    if (g_off != INT64_MAX && end >= 0 && end < (int64_t)kTileBytes) {
      if (!staged) {
        win_global = true;
      } else {
        const uint32_t sb = (uint32_t)(end - 7 + 16);  // window start in stage bytes: 9 ..
        const uint32_t w = sb >> 2, sh = 8u * (sb & 3u);
        const uint32_t u0 = stage[w], u1 = stage[w + 1], u2 = (sb & 3u) ? stage[w + 2] : 0u;
        win_lo = __funnelshift_r(u0, u1, sh);
        win_hi = __funnelshift_r(u1, u2, sh);
      }
    }
  };


  for (uint32_t i = 0; i < n_tiles; ++i) {
    // ---- stream the tile (plain `lookup` over the concatenation) ----------
    if (i + 2 < n_tiles) issue(i + 2);
    cp_async_commit();
    cp_async_wait<kStages - 1>();
    __syncwarp();  // every lane's part of tile i is in its slot
    stage = ring + rd * kSlotWords;
    err_words = stage + 4;
    uint4 d[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) d[r] = reinterpret_cast<const uint4*>(stage + 4)[r * kLanes + lane];
    const int64_t tile_lo = vbase + (int64_t)((t0 + i) * kTileBytes);
    take_windows(tile_lo, true);
    bool staged = true;  // the stage still holds this tile
    uint32_t e[ROWS / 2][8];
    check_tile<ROWS, kBatchQuads<ROWS>>(d, carry, lane, merge_sel, e);
    uint32_t any_err = 0;
#pragma unroll
    for (int p = 0; p < ROWS / 2; ++p)
#pragma unroll
      for (int m = 0; m < 8; ++m) any_err |= e[p][m];

    // ---- charge streamed errors to strings (only where errors exist) -----
    // Boundaries before next_group lie before this tile, so a position p of
    // the tile belongs to string next_group - 1 + (number of the open group's
    // boundaries <= p), one ballot over g_off, unless p lies past the group's
    // last boundary (then a binary search).  The warp takes the error bytes
    // one at a time: they go through shared memory so that each lane walks
    // its own in one rolled loop.
    if (__any_sync(kFull, any_err != 0)) {
      staged = false;
      __syncwarp();  // every lane has taken its windows from the stage
      static_assert(ROWS / 2 * 8 <= 32, "one bit per error word");
      uint32_t nonzero = 0;  // bit w: error word w of this lane is non-zero
#pragma unroll
      for (int pr = 0; pr < ROWS / 2; ++pr)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          err_words[(pr * 8 + m) * kLanes + lane] = e[pr][m];
          nonzero |= (e[pr][m] != 0 ? 1u : 0u) << (pr * 8 + m);
        }
      __syncwarp();
      const int gsize = next_group < b1 ? (int)(group_last - next_group + 1) : 0;
      // the next group's size (its offsets g_nxt are in the lanes already)
      const int nsize = gsize > 0 && group_last + 1 < b1
                            ? (int)((group_last + 1 + kLanes < b1 ? group_last + 1 + kLanes : b1) -
                                    (group_last + 1))
                            : 0;
      const int64_t group_last_off = __shfl_sync(kFull, g_off, gsize > 0 ? gsize - 1 : 0);
      int k = 0, byte = 0;
      uint32_t bits = 0;
      for (;;) {
        // this lane's next error byte, if any
        while (bits == 0 && nonzero != 0) {
          k = __ffs(nonzero) - 1;
          nonzero &= nonzero - 1;
          bits = err_words[k * kLanes + lane];
        }
        int64_t p = INT64_MAX;
        if (bits != 0) {
          byte = (__ffs(bits) - 1) >> 3;
          // row pairs: bytes `byte` and byte + 2 are positions 2m and 2m+1
          // of one row, and the first decides for both (the same string, or
          // 2m+1 starts one, and a string's first three bytes are the head
          // check's); in a quad word every byte is a row of its own
          if constexpr (kBatchQuads<ROWS>) bits &= ~(0xFFu << (8 * byte));
          else bits &= ~(0x00FF00FFu << (8 * byte));
          p = tile_lo + (int64_t)interleaved_position<ROWS, kBatchQuads<ROWS>>(k >> 3, k & 7, byte, lane);
        }
        uint32_t pending = __ballot_sync(kFull, p != INT64_MAX);
        if (pending == 0) break;
        while (pending != 0) {
          const int src = __ffs(pending) - 1;
          pending &= pending - 1;
          const int64_t q = __shfl_sync(kFull, p, src);
          const int cnt = __popc(__ballot_sync(kFull, g_off <= q));
          const int64_t lo_cnt = __shfl_sync(kFull, g_off, cnt > 0 ? cnt - 1 : 0);
          // past the open group: the next group's offsets, before a search
          const int cnt2 = __popc(__ballot_sync(kFull, g_nxt <= q));
          const int64_t lo_cnt2 = __shfl_sync(kFull, g_nxt, cnt2 > 0 ? cnt2 - 1 : 0);
          if (lane == src) {
            int64_t own, o_lo, o_hi;
            if (cnt < gsize || gsize == 0) {
              own = next_group - 1 + cnt;
              o_lo = cnt > 0 ? lo_cnt : prev_off;
              o_hi = INT64_MAX;  // the next boundary lies past q
            } else if (cnt2 < nsize) {
              own = group_last + cnt2;
              o_lo = cnt2 > 0 ? lo_cnt2 : group_last_off;
              o_hi = INT64_MAX;
            } else {
              own = last_at_most(offsets, group_last, own_hi + 1, q);
              o_lo = own >= 0 && own <= count ? offsets[own] : 0;
              o_hi = own >= 0 && own < count ? offsets[own + 1] : 0;
            }
            const bool charged = own >= 0 && own < count && q - o_lo >= 3 && q < o_hi;
            if (charged) charge<LOCATE>(out_valid, out_err, own, q - o_lo);
            if constexpr (kBatchQuads<ROWS>) {
              // the next positions of the row are bytes `byte` of the next
              // words: p + 1 is the same string or lies in the first three
              // bytes of the next (the head check's), and so are p + 2 and
              // p + 3 once p's string is charged
              const int kk = k & 15;
              const int last = charged ? 3 : 1;
              for (int t = 1; t <= last && kk + t < 16; ++t)
                err_words[(k + t) * kLanes + lane] &= ~(0xFFu << (8 * byte));
            }
          }
        }
      }
      __syncwarp();
    }

    // ---- boundaries: exact head and tail checks, 32 at a time ------------
    // Lane k takes boundary j = next_group + k at o_j: the tail of string
    // j-1, [o_{j-1}, o_j), and the head of string j, [o_j, o_{j+1}).  The
    // neighbouring offsets come from the neighbouring lanes.
    while (i >= due || (i + 1 == n_tiles && next_group < b1)) {
      const int64_t j = next_group + lane;
      const bool act = lane <= (int)(group_last - next_group);
      const int64_t oj = g_off;
      int64_t o_prev = __shfl_up_sync(kFull, oj, 1);
      int64_t o_next = __shfl_down_sync(kFull, oj, 1);
      const int64_t after_group = __shfl_sync(kFull, g_nxt, 0);  // offsets[group_last + 1]
      if (lane == 0) o_prev = prev_off;
      if (act && j == group_last && j < count)
        o_next = group_last + 1 < b1 ? after_group : offsets[j + 1];
      if (act) {
        const int64_t lo = j >= 1 ? o_prev : oj;
        const int64_t hi = j < count ? o_next : oj;
        uint32_t w_tail, w_head;  // bytes [o_j - 4, o_j) and [o_j, o_j + 4), in [lo, hi)
        if (win_global || oj + 3 >= tile_lo + (int64_t)kTileBytes) {
          // window replaced in the stage, or ending past this warp's last tile
          gather8(data, oj - 4, lo, hi, w_tail, w_head);
        } else {
          const int64_t x = oj - 4;
          const int ka = (int)((lo > x ? lo : x) - x), kb = (int)((hi < x + 8 ? hi : x + 8) - x);
          w_tail = win_lo & keep_bytes(ka, kb);
          w_head = win_hi & keep_bytes(ka - 4, kb - 4);
        }
        WordLut tail, head;
        lut_pair(w_tail, w_head, tail, head);
        if (j >= 1) {  // positions o_j .. o_j+3 after string j-1 (virtual zeros)
          const uint32_t te = word_error(tail, ascii_lut());
          if (te != 0) charge<LOCATE>(out_valid, out_err, j - 1, oj - lo + ((__ffs(te) - 1) >> 3));
        }
        if (j < count) {  // positions o_j .. o_j+3 of string j (zeros before it)
          const uint32_t he = word_error(ascii_lut(), head);
          if (he != 0) charge<LOCATE>(out_valid, out_err, j, (__ffs(he) - 1) >> 3);
        }
      }
      prev_off = __shfl_sync(kFull, g_off, (int)(group_last - next_group));
      next_group = group_last + 1;
      open_group();
      take_windows(tile_lo, staged);
    }
    // the 8 bytes before the next tile: this tile's last 8 (lane 31, last
    // row), into the next slot's header
    rd = rd + 1 == kStages ? 0 : rd + 1;
    if (lane == kLanes - 1) {
      ring[rd * kSlotWords + 2] = d[ROWS - 1].z;
      ring[rd * kSlotWords + 3] = d[ROWS - 1].w;
    }
    __syncwarp();
  }
  cp_async_wait<0>();
}

template <int ROWS, bool LOCATE>
__global__ void __launch_bounds__(kBlockThreads)
    batch_kernel(const uint8_t* __restrict__ data, const int64_t* __restrict__ offsets,
                 int64_t count, uint8_t* __restrict__ out_valid, utf8_error_info* out_err) {
  batch_body<ROWS, LOCATE>(data, offsets, count, out_valid, out_err);
}

// The same pass with its arguments read from a device descriptor when it
// runs, so that one captured graph serves any batch written into it.
template <int ROWS>
__global__ void __launch_bounds__(kBlockThreads, 2) batch_desc_kernel(const utf8_batch_desc* desc) {
  const utf8_batch_desc d = *desc;
  if (d.count <= 0) return;
  batch_body<ROWS, false>(d.data, d.offsets, d.count, d.out_valid, nullptr);
}

// Sets the descriptor's count flags to 1 (the batch pass only clears them).
__global__ void set_flags_desc_kernel(const utf8_batch_desc* desc) {
  const int64_t count = desc->count;
  uint8_t* out = desc->out_valid;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    out[i] = 1;
}

template <int ROWS, bool LOCATE = false>
static cudaError_t launch_batch_rows(const uint8_t* data, const int64_t* offsets, int64_t count,
                                     uint8_t* out_valid, int blocks_per_sm, int sm_count,
                                     cudaStream_t st, utf8_error_info* out_err = nullptr) {
  const unsigned grid = (unsigned)(sm_count * blocks_per_sm);
  batch_kernel<ROWS, LOCATE><<<grid, kBlockThreads, batch_smem_bytes<ROWS>(), st>>>(
      data, offsets, count, out_valid, out_err);
  return cudaGetLastError();
}

cudaError_t launch_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                         uint8_t* out_valid, const LaunchCfg& cfg, int sm_count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out_valid, 1, (size_t)count, st);
  if (e != cudaSuccess) return e;
  switch (cfg.batch_rows) {
    case 8: return launch_batch_rows<8>(data, offsets, count, out_valid, cfg.batch_blocks_per_sm,
                                        sm_count, st);
    case 4: return launch_batch_rows<4>(data, offsets, count, out_valid, cfg.batch_blocks_per_sm,
                                        sm_count, st);
    default: return launch_batch_rows<2>(data, offsets, count, out_valid, cfg.batch_blocks_per_sm,
                                         sm_count, st);
  }
}

cudaError_t launch_batch_desc(const utf8_batch_desc* desc, const LaunchCfg& cfg, int sm_count,
                              cudaStream_t st) {
  set_flags_desc_kernel<<<(unsigned)(sm_count * 4), 256, 0, st>>>(desc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)(sm_count * cfg.batch_blocks_per_sm);
  switch (cfg.batch_rows) {
    case 8: batch_desc_kernel<8><<<grid, kBlockThreads, batch_smem_bytes<8>(), st>>>(desc); break;
    case 4: batch_desc_kernel<4><<<grid, kBlockThreads, batch_smem_bytes<4>(), st>>>(desc); break;
    default: batch_desc_kernel<2><<<grid, kBlockThreads, batch_smem_bytes<2>(), st>>>(desc); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_first_errors(const uint8_t* data, const int64_t* offsets, int64_t count,
                                      utf8_error_info* out, const LaunchCfg& cfg, int sm_count,
                                      cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  switch (cfg.batch_rows) {
    case 8: return launch_batch_rows<8, true>(data, offsets, count, nullptr,
                                              cfg.batch_blocks_per_sm, sm_count, st, out);
    case 4: return launch_batch_rows<4, true>(data, offsets, count, nullptr,
                                              cfg.batch_blocks_per_sm, sm_count, st, out);
    default: return launch_batch_rows<2, true>(data, offsets, count, nullptr,
                                               cfg.batch_blocks_per_sm, sm_count, st, out);
  }
}

}  // namespace utf8gpu

namespace utf8gpu {

// Offsets well-formed: offsets[0] >= 0 and non-decreasing; clears *out_ok
// otherwise (the caller sets it to 1).
__global__ void check_offsets_kernel(const int64_t* __restrict__ offsets, int64_t count,
                                     uint8_t* out_ok) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= count; i += stride) {
    const int64_t o = offsets[i];
    if (i == 0 && o < 0) bad = true;
    if (i < count && o > offsets[i + 1]) bad = true;
  }
  if (bad) *out_ok = 0;
}

cudaError_t launch_check_offsets(const int64_t* offsets, int64_t count, uint8_t* out_ok,
                                 int sm_count, cudaStream_t st) {
  const int64_t blocks = (count + 1 + 255) / 256;
  const int64_t cap = (int64_t)sm_count * 8;
  check_offsets_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, st>>>(offsets, count,
                                                                               out_ok);
  return cudaGetLastError();
}

}  // namespace utf8gpu

namespace utf8gpu {

// Lets every batch kernel of `ROWS` rows use its rings' shared memory.
template <int ROWS>
static cudaError_t allow_batch_smem() {
  const int smem = batch_smem_bytes<ROWS>();
  cudaError_t e = cudaSuccess;
  const auto allow = [&](const void* f) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
  };
  allow(reinterpret_cast<const void*>(batch_kernel<ROWS, false>));
  allow(reinterpret_cast<const void*>(batch_kernel<ROWS, true>));
  allow(reinterpret_cast<const void*>(batch_desc_kernel<ROWS>));
  return e;
}

// Resident CTAs per SM of the batch kernels at `rows` rows, with their rings
// (0 when this device cannot give them the shared memory).
int batch_blocks_per_sm(int rows) {
  int n = 0;
  cudaError_t e;
  switch (rows) {
    case 8:
      e = allow_batch_smem<8>();
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<8, false>, kBlockThreads,
                                                          batch_smem_bytes<8>());
      break;
    case 4:
      e = allow_batch_smem<4>();
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<4, false>, kBlockThreads,
                                                          batch_smem_bytes<4>());
      break;
    default:
      e = allow_batch_smem<2>();
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<2, false>, kBlockThreads,
                                                          batch_smem_bytes<2>());
      break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace utf8gpu

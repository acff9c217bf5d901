// Warp-cooperative lower bound over a sorted int64 array: the narrowing step
// as plain host/device functions of the 32 probe results, so that the same
// code is checked exhaustively on the host.
#pragma once
#include <stdint.h>

namespace utf8gpu {

// Range [lo, hi]: the answer (first index j in [lo, hi) with a[j] >= target,
// or hi if there is none) lies in it.  One step probes j_k = lo + k * step
// (k = 0..31; a probe at or past hi counts as true) and narrows the range from
// the probe mask (bit k = probe k true).
struct LbRange {
  int64_t lo, hi;
};

__host__ __device__ inline int64_t lb_step(int64_t lo, int64_t hi) {
  return (hi - lo + 31) / 32;
}

__host__ __device__ inline LbRange lb_narrow(int64_t lo, int64_t hi, int64_t step,
                                             uint32_t mask) {
  LbRange r;
  if (mask == 0) {  // every probe false: the answer is after the last probe
    r.lo = lo + 31 * step + 1;
    r.hi = hi;
  } else {
    int f = 0;
    while (!((mask >> f) & 1u)) ++f;  // first true probe
    const int64_t jf = lo + (int64_t)f * step;
    r.lo = f == 0 ? lo : lo + (int64_t)(f - 1) * step + 1;
    r.hi = jf < hi ? jf : hi;
  }
  if (r.lo > r.hi) r.lo = r.hi;
  return r;
}

// Last round, hi - lo <= 32: probe k is lo + k.
__host__ __device__ inline int64_t lb_final(int64_t lo, int64_t hi, uint32_t mask) {
  for (int k = 0; k < 32 && lo + k < hi; ++k)
    if ((mask >> k) & 1u) return lo + k;
  return hi;
}

// Last j in [lo, hi) with a[j] <= p, or lo - 1 if there is none.
__host__ __device__ inline int64_t last_at_most(const int64_t* a, int64_t lo, int64_t hi,
                                                int64_t p) {
  int64_t x = lo - 1, y = hi;  // a[x] <= p and a[y] > p, virtually
  while (y - x > 1) {
    const int64_t m = x + (y - x) / 2;
    if (a[m] <= p) x = m; else y = m;
  }
  return x;
}

}  // namespace utf8gpu

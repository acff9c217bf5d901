// Host check of the batch kernel's search helpers (search.cuh), compiled
// with g++ as plain C++: the warp's 32 probes are evaluated on the host.
#define __host__
#define __device__
#include <stdint.h>
#include <stdio.h>
#include <algorithm>
#include <random>
#include <vector>
#include "search.cuh"

using namespace utf8gpu;

static int64_t warp_lower_bound_host(const std::vector<int64_t>& a, int64_t lo, int64_t hi,
                                     int64_t target, int* rounds) {
  *rounds = 0;
  while (hi - lo > 32) {
    const int64_t step = lb_step(lo, hi);
    uint32_t mask = 0;
    for (int k = 0; k < 32; ++k) {
      const int64_t j = lo + k * step;
      if (j >= hi || a[j] >= target) mask |= 1u << k;
    }
    const LbRange r = lb_narrow(lo, hi, step, mask);
    if (r.lo < lo || r.hi > hi || r.hi - r.lo >= hi - lo) return -999;  // must shrink inside
    lo = r.lo;
    hi = r.hi;
    if (++*rounds > 64) return -998;
  }
  uint32_t mask = 0;
  for (int k = 0; k < 32; ++k) {
    const int64_t j = lo + k;
    if (j >= hi || a[j] >= target) mask |= 1u << k;
  }
  return lb_final(lo, hi, mask);
}

// The batch kernel's two searches in one loop (warp_lower_bound2): both
// ranges are probed each round, a range stops narrowing once it is at most
// 32 wide, and both finish with one more probe round.
static void warp_lower_bound2_host(const std::vector<int64_t>& a, int64_t hi, int64_t ta,
                                   int64_t tb, int64_t* ra, int64_t* rb, int* rounds) {
  int64_t lo_a = 0, hi_a = hi, lo_b = 0, hi_b = hi;
  *rounds = 0;
  auto probe = [&](int64_t lo, int64_t h, int64_t step, int64_t t) {
    uint32_t mask = 0;
    for (int k = 0; k < 32; ++k) {
      const int64_t j = lo + k * step;
      if (j >= h || a[j] >= t) mask |= 1u << k;
    }
    return mask;
  };
  while (hi_a - lo_a > 32 || hi_b - lo_b > 32) {
    if (hi_a - lo_a > 32) {
      const int64_t s = lb_step(lo_a, hi_a);
      const LbRange r = lb_narrow(lo_a, hi_a, s, probe(lo_a, hi_a, s, ta));
      lo_a = r.lo;
      hi_a = r.hi;
    }
    if (hi_b - lo_b > 32) {
      const int64_t s = lb_step(lo_b, hi_b);
      const LbRange r = lb_narrow(lo_b, hi_b, s, probe(lo_b, hi_b, s, tb));
      lo_b = r.lo;
      hi_b = r.hi;
    }
    if (++*rounds > 64) break;
  }
  *ra = lb_final(lo_a, hi_a, probe(lo_a, hi_a, 1, ta));
  *rb = lb_final(lo_b, hi_b, probe(lo_b, hi_b, 1, tb));
}

int main() {
  std::mt19937_64 rng(20100309);
  int64_t checks = 0, bad = 0;
  std::vector<int64_t> sizes;
  for (int64_t n = 0; n <= 300; ++n) sizes.push_back(n);
  for (int64_t n : {1023, 1024, 1025, 32767, 32768, 32769, 65536, 65537, 1000001}) sizes.push_back(n);
  for (int64_t n : sizes) {
    std::vector<int64_t> a(n);
    int64_t v = 0;
    for (int64_t i = 0; i < n; ++i) { v += (int64_t)(rng() % 4); a[i] = v; }  // sorted, with repeats
    std::vector<int64_t> targets = {-1, 0, v, v + 1, v + 100};
    for (int t = 0; t < (n < 400 ? 200 : 50); ++t) targets.push_back((int64_t)(rng() % (uint64_t)(v + 3)) - 1);
    for (int64_t i = 0; i < n && i < 64; ++i) targets.push_back(a[n - 1 - i]);
    for (int64_t target : targets) {
      int rounds = 0;
      const int64_t want = std::lower_bound(a.begin(), a.end(), target) - a.begin();
      const int64_t got = warp_lower_bound_host(a, 0, n, target, &rounds);
      ++checks;
      if (got != want) {
        if (bad < 10) printf("lower_bound n=%lld target=%lld got=%lld want=%lld\n",
                             (long long)n, (long long)target, (long long)got, (long long)want);
        ++bad;
      }
      // both searches of a warp at once: this target and a second one
      const int64_t target_b = target + (int64_t)(rng() % 5000);
      int64_t ra = 0, rb = 0;
      warp_lower_bound2_host(a, n, target, target_b, &ra, &rb, &rounds);
      const int64_t want_b = std::lower_bound(a.begin(), a.end(), target_b) - a.begin();
      ++checks;
      if (ra != want || rb != want_b || rounds > 8) {
        if (bad < 10) printf("lower_bound2 n=%lld targets=%lld,%lld got=%lld,%lld want=%lld,%lld\n",
                             (long long)n, (long long)target, (long long)target_b, (long long)ra,
                             (long long)rb, (long long)want, (long long)want_b);
        ++bad;
      }
      // last_at_most over a sub-range
      const int64_t lo = n ? (int64_t)(rng() % (uint64_t)n) : 0;
      const int64_t hi = lo + (n - lo ? (int64_t)(rng() % (uint64_t)(n - lo + 1)) : 0);
      int64_t want2 = lo - 1;
      for (int64_t j = lo; j < hi; ++j) if (a[j] <= target) want2 = j;
      const int64_t got2 = last_at_most(a.data(), lo, hi, target);
      ++checks;
      if (got2 != want2) {
        if (bad < 10) printf("last_at_most n=%lld [%lld,%lld) p=%lld got=%lld want=%lld\n",
                             (long long)n, (long long)lo, (long long)hi, (long long)target,
                             (long long)got2, (long long)want2);
        ++bad;
      }
    }
  }
  printf("%lld checks, %lld bad\n", (long long)checks, (long long)bad);
  return bad ? 1 : 0;
}

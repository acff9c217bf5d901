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

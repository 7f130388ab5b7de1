// Host-side check of the walk's division by invariant integers (FastDiv in
// spmc_device.cuh): the multiply-shift quotient equals n / d for divisors of
// every size, numerators at the edges of each quotient step and random ones.
// Built by nvcc and run on the host cores only (no device code is launched).
#include <cstdio>
#include <cstdint>
#include <random>

#include "../paper_2608_22190_b300/csrc/spmc_device.cuh"

int main() {
  std::mt19937_64 g(7);
  long long bad = 0, tests = 0;
  auto check = [&](const spmc::FastDiv& f, uint32_t n) {
    ++tests;
    if (f.div(n) != n / f.d) {
      if (bad < 10) std::printf("d = %u n = %u: %u != %u\n", f.d, n, f.div(n), n / f.d);
      ++bad;
    }
  };
  // every divisor below 4096 against every numerator below 2^16, and the top of the range
  for (uint32_t d = 1; d < 4096; ++d) {
    const spmc::FastDiv f(d);
    for (uint32_t n = 0; n < 65536; ++n) check(f, n);
    for (uint32_t k = 0; k < 64; ++k) check(f, 0xffffffffu - k);
  }
  // random divisors of every bit length, numerators next to multiples of d and random
  for (int i = 0; i < 100000; ++i) {
    uint32_t d = (uint32_t)(g() >> (32 + g() % 32));
    if (d == 0) d = 1;
    const spmc::FastDiv f(d);
    for (int k = 0; k < 8; ++k) {
      const uint64_t q = g() % (0xffffffffull / d + 1);
      const uint64_t base = q * d;
      for (int o = -1; o <= 1; ++o) {
        const int64_t n = (int64_t)base + o;
        if (n >= 0 && n <= 0xffffffffll) check(f, (uint32_t)n);
      }
      check(f, (uint32_t)g());
    }
  }
  std::printf("%lld checks, %lld wrong\n", tests, bad);
  return bad == 0 ? 0 : 1;
}

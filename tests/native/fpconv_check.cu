// Host check of the integer-only binary32 <-> binary64 conversions against the
// compiler's conversions: every binary32 value for f2d_exact; for d2f_rn every
// exponent around the binary32 range with random fractions, the exact halfway
// patterns (ties to even) in the normal and subnormal ranges, and random bit
// patterns.  Prints "ok <counts>" or the first mismatch and exits non-zero.
#include <cmath>
#include <cstdio>
#include <random>

#include "fpconv.cuh"

using namespace pbs;

static bool same_f(float a, float b) { return (std::isnan(a) && std::isnan(b)) || bits_of(a) == bits_of(b); }
static bool same_d(double a, double b) { return (std::isnan(a) && std::isnan(b)) || bits_of(a) == bits_of(b); }

static int check_d2f(double d, long& n) {
  ++n;
  const float want = (float)d, got = d2f_rn(d);
  if (!same_f(want, got)) {
    std::printf("d2f mismatch: d bits %016llx want %08x got %08x\n", (unsigned long long)bits_of(d), bits_of(want),
                bits_of(got));
    return 1;
  }
  return 0;
}

int main() {
  long nf = 0, nd = 0;
  for (uint64_t u = 0; u <= 0xFFFFFFFFull; ++u) {
    const float f = float_of((uint32_t)u);
    ++nf;
    if (!same_d((double)f, f2d_exact(f))) {
      std::printf("f2d mismatch: f bits %08x\n", (unsigned)u);
      return 1;
    }
  }
  std::mt19937_64 rng(12345);
  for (int E = -1100; E <= 1100; ++E) {
    if (E < -1075 && E != -1100) continue;
    const int e = E + 1023;
    for (int t = 0; t < 4000; ++t) {
      const uint64_t m = rng() & 0xFFFFFFFFFFFFFull, sgn = (rng() & 1ull) << 63;
      const uint64_t ef = e < 0 ? 0 : (e > 2047 ? 2047 : (uint64_t)e);
      if (check_d2f(double_of(sgn | (ef << 52) | m), nd)) return 1;
    }
    if (E >= -160 && E <= 130 && E + 1023 > 0) {
      // halfway and neighbouring patterns of the bits binary32 drops at this exponent
      const int dropped = E >= -126 ? 29 : -E - 97 + 0;  // fraction bits below the kept ones
      for (int k = 0; k < 200; ++k) {
        const uint64_t keep = rng() & 0xFFFFFFFFFFFFFull;
        for (int dlt = -1; dlt <= 1; ++dlt) {
          uint64_t m;
          if (dropped >= 52) {
            m = (uint64_t)((int64_t)(dlt < 0 ? 0 : dlt));
          } else {
            const uint64_t mask = (1ull << dropped) - 1ull, half = 1ull << (dropped - 1);
            m = ((keep & ~mask) | ((half + (uint64_t)(int64_t)dlt) & mask)) & 0xFFFFFFFFFFFFFull;
          }
          if (check_d2f(double_of(((uint64_t)(E + 1023) << 52) | m), nd)) return 1;
          if (check_d2f(double_of((1ull << 63) | ((uint64_t)(E + 1023) << 52) | m), nd)) return 1;
        }
      }
    }
  }
  for (long t = 0; t < 20000000; ++t)
    if (check_d2f(double_of(rng()), nd)) return 1;
  const double specials[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 3.4028234663852886e38, 3.4028235677973366e38,
                             3.4028235677973362e38, 1.1754943508222875e-38, 1.1754942106924411e-38,
                             1.401298464324817e-45, 7.006492321624085e-46, 7.006492321624087e-46,
                             2.1019476964872256e-45, 1e-300, -1e300};
  for (double d : specials)
    if (check_d2f(d, nd)) return 1;
  std::printf("ok %ld %ld\n", nf, nd);
  return 0;
}

// Host-side check of the integer-pipe float/double conversions of
// mto_common.cuh against the C casts (compiled by nvcc as host code).
// Prints "ok <count>" or the first mismatch and exits non-zero.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "mto_common.cuh"

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {  // xorshift64*
  state ^= state >> 12;
  state ^= state << 25;
  state ^= state >> 27;
  return state * 0x2545F4914F6CDD1Dull;
}

static int check_d2f(double d) {
  const float want = (float)d;
  const float got = mto::d2f_rn(d);
  if (std::isnan(want)) return std::isnan(got) ? 0 : 1;
  // Below the float normal range the integer conversion gives signed zero.
  if (std::fabs(want) < 1.17549435e-38f) return (got == 0.0f && std::signbit(got) == std::signbit(d)) ? 0 : 1;
  return mto::bits_of(got) == mto::bits_of(want) ? 0 : 1;
}

int main() {
  long long n = 0;
  // Random bit patterns over the whole double range, values near float
  // rounding boundaries, and special values.
  for (int t = 0; t < 4000000; ++t) {
    double d;
    uint64_t b = next_u64();
    if (t % 4 == 1) {
      // exponent inside the float range
      b = (b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(896 + 1 + (next_u64() % 254)) << 52);
    } else if (t % 4 == 2) {
      // a float value plus a tie or near-tie in the dropped bits
      const uint64_t fb = ((uint64_t)(896 + 1 + (next_u64() % 254)) << 52) | ((next_u64() & 0x7FFFFFull) << 29);
      const uint64_t tails[] = {0x10000000ull, 0x0FFFFFFFull, 0x10000001ull, 0x1FFFFFFFull, 0ull};
      b = fb | tails[next_u64() % 5] | (next_u64() & 0x8000000000000000ull);
    } else if (t % 4 == 3) {
      b = (b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(896 - 30 + (next_u64() % 320)) << 52);
    }
    std::memcpy(&d, &b, 8);
    if (check_d2f(d)) {
      std::printf("d2f mismatch at %.17g (bits %016llx): got %.9g want %.9g\n", d, (unsigned long long)b,
                  mto::d2f_rn(d), (float)d);
      return 1;
    }
    ++n;
  }
  const double specials[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                             1e39, -1e39, INFINITY, -INFINITY, NAN, 1.1754943508222875e-38,
                             1.1754942e-38, 5e-324, 0.1, 1.0 / 3.0};
  for (double d : specials) {
    if (check_d2f(d)) {
      std::printf("d2f mismatch at special %.17g\n", d);
      return 1;
    }
    ++n;
  }
  // float -> double: exact for every normal float, signed zero for subnormals.
  for (uint64_t u = 0; u < (1ull << 32); u += 997) {
    const float f = mto::float_of((unsigned)u);
    const double got = mto::f2d_exact(f);
    const bool sub = std::fpclassify(f) == FP_SUBNORMAL;
    bool ok;
    if (std::isnan(f)) ok = std::isnan(got);
    else if (sub) ok = got == 0.0 && std::signbit(got) == std::signbit(f);
    else ok = mto::bits_of(got) == mto::bits_of((double)f);
    if (!ok) {
      std::printf("f2d mismatch at bits %08x\n", (unsigned)u);
      return 1;
    }
    ++n;
  }
  std::printf("ok %lld\n", n);
  return 0;
}

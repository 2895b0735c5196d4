// Host-side check of the integer-only conversions and comparisons of the device code: fixed_to_double
// (the exact fixed-point sums, the 53-bit uniforms, counts) must equal static_cast<double>(v) * 2^-frac
// for edge cases and random 64-bit values; f32_of_double must equal static_cast<float> and
// dbl_gt / dbl_lt / dbl_is_zero / dbl_finite the floating-point comparisons on random bit patterns,
// specials and neighbours of the constants compared against.
// Usage: fixed_to_double_check N -> prints "n mismatches"; exit status 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#include "duwp_dsmath.cuh"

using namespace duwp;

static bool same(double a, double b) { return std::memcmp(&a, &b, 8) == 0; }

int main(int argc, char **argv)
{
    const long n = argc > 1 ? std::atol(argv[1]) : 1000000;
    std::mt19937_64 rng(12345);
    long bad = 0, tot = 0;
    auto check = [&](int64_t v, int frac) {
        const double want = static_cast<double>(v) * std::ldexp(1.0, -frac);
        const double got = fixed_to_double(v, frac);
        ++tot;
        if (!same(want, got)) {
            if (bad < 10) std::printf("mismatch v=%lld frac=%d want=%.17g got=%.17g\n", (long long)v, frac, want, got);
            ++bad;
        }
    };
    const int fracs[3] = {0, 32, 40};
    for (int f : fracs) {
        // powers of two, their neighbours, and the tie cases around 2^53 .. 2^62
        for (int k = 0; k < 63; ++k) {
            const int64_t p = int64_t(1) << k;
            for (int64_t d = -3; d <= 3; ++d) { check(p + d, f); check(-(p + d), f); }
        }
        for (int sh = 1; sh <= 10; ++sh)
            for (int64_t q = 0; q < 64; ++q) {
                const int64_t base = (int64_t(1) << 52) + q;
                const int64_t v = (base << sh) + (int64_t(1) << (sh - 1));   // exact ties
                check(v, f); check(-v, f); check(v + 1, f); check(v - 1, f);
            }
        check(INT64_MAX, f);
        check(-INT64_MAX, f);
    }
    for (long i = 0; i < n; ++i) {
        const int bitsz = 1 + static_cast<int>(rng() % 63);
        int64_t v = static_cast<int64_t>(rng() >> (64 - bitsz));
        if (rng() & 1) v = -v;
        check(v, fracs[i % 3]);
    }
    // double -> float and the comparisons, on random bit patterns of every exponent, ties, specials
    auto checkf = [&](double x) {
        const float want = static_cast<float>(x), got = f32_of_double(x);
        ++tot;
        if (std::memcmp(&want, &got, 4) != 0 && !(std::isnan(want) && std::isnan(got))) {
            if (bad < 10) std::printf("f32 mismatch x=%.17g want=%.9g got=%.9g\n", x, want, got);
            ++bad;
        }
        const double cs[4] = {0.0, 1e-30, 1e8, 1e30};
        for (double c : cs) {
            ++tot;
            if (dbl_gt(x, c) != (x > c) || (c > 0.0 && dbl_lt(x, c) != (x < c))) {
                if (bad < 10) std::printf("compare mismatch x=%.17g c=%g\n", x, c);
                ++bad;
            }
        }
        ++tot;
        if (dbl_is_zero(x) != (x == 0.0) || dbl_finite(x) != static_cast<bool>(std::isfinite(x))) {
            if (bad < 10) std::printf("zero/finite mismatch x=%.17g\n", x);
            ++bad;
        }
    };
    for (long i = 0; i < n; ++i) {
        uint64_t b = rng();
        if (i % 3 == 0) b = (b & 0x800fffffffffffffull) | (static_cast<uint64_t>(1023 - 130 + rng() % 262) << 52);
        if (i % 7 == 0) b = (b & ~0x1fffffffull) | 0x10000000ull;                 // float rounding ties
        if (i % 11 == 0) b |= 0x000fffffe0000000ull;                                 // carries
        double x;
        std::memcpy(&x, &b, 8);
        checkf(x);
    }
    const double sp[] = {0.0, -0.0, 1e-30, 1e30, 1e8, std::nextafter(1e-30, 0.0), std::nextafter(1e-30, 1.0),
                         std::nextafter(1e30, 0.0), std::nextafter(1e30, 2e30), std::nextafter(1e8, 0.0),
                         std::nextafter(1e8, 2e8), HUGE_VAL, -HUGE_VAL, std::nan(""), -std::nan(""),
                         3.4028235677973366e38, 3.4028235677973362e38, 1.1754943508222875e-38,
                         1.1754942807573643e-38, 5e-324, -5e-324};
    for (double x : sp) checkf(x);
    std::printf("%ld %ld\n", tot, bad);
    return bad ? 1 : 0;
}

// Host-side check of fixed_to_double (the integer-only conversion of the exact fixed-point sums):
// for edge cases and random 64-bit values it must equal static_cast<double>(v) * 2^-frac.
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
    std::printf("%ld %ld\n", tot, bad);
    return bad ? 1 : 0;
}

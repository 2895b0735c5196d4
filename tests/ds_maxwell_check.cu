// Host-side check of the double-single Maxwellian sampling of single-precision records: for random
// draws and cell states, whenever ds_maxwell reports success its floats must equal the
// single-precision rounding of the double-precision evaluation of Eq. (maxsample) by the Box-Muller
// pair, xi_x = U + (sqrt(2RT) cos(2 pi r1)) sqrt(-log(1 - r2)), xi_y = V + (sqrt(2RT) sin(2 pi r1))
// sqrt(-log(1 - r2)), xi_z = W + (sqrt(2RT) cos(2 pi r3)) sqrt(-log(1 - r4)), with r1..r4 the 53-bit
// uniforms of the draw words; the fallback must stay rare.  Also checks -log(1 - u) against long double.
// Usage: ds_maxwell_check N  -> prints "n fallbacks mismatches max_log_rel_err"; exit 1 on a mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#include "duwp_dsmath.cuh"

using namespace duwp;

static double u53_host(uint32_t a, uint32_t b)
{
    const uint64_t m = (static_cast<uint64_t>(a) << 21) ^ static_cast<uint64_t>(b >> 11);
    return static_cast<double>(m) * 0x1p-53;
}

int main(int argc, char **argv)
{
    float4 turn[kTurnTable];
    for (int k = 0; k < kTurnTable; ++k) {
        const long double ang = 2.0L * 3.14159265358979323846264338327950288L * k / kTurnTable;
        const double c = static_cast<double>(cosl(ang)), s = static_cast<double>(sinl(ang));
        const float ch = static_cast<float>(c), sh = static_cast<float>(s);
        turn[k] = make_float4(ch, static_cast<float>(c - ch), sh, static_cast<float>(s - sh));
    }
    float4 logt[kLogTable];
    for (int k = 0; k < kLogTable; ++k) {
        const long double F = (long double)(1024 + k - kLogCenter) / 1024.0L;
        const long double inv = 1.0L / F, lg = logl(F);
        const float ih = static_cast<float>(inv), lh = static_cast<float>(lg);
        logt[k] = make_float4(ih, static_cast<float>(inv - ih), lh, static_cast<float>(lg - lh));
    }
    std::mt19937_64 rng(2306);
    // the integer double -> double-single conversion against the double-precision one, on random bit
    // patterns over its whole exponent range (ties and carries included by the low bits chosen)
    for (long t = 0; t < 2000000; ++t) {
        uint64_t bits = rng();
        const uint64_t e = static_cast<uint64_t>(1023 - 70 + static_cast<int>(rng() % 170));
        bits = (bits & 0x800fffffffffffffull) | (e << 52);
        if (t % 4 == 1) bits = (bits & ~0x1fffffffull) | 0x10000000ull;            // exact tie
        if (t % 4 == 2) bits |= 0x000fffffe0000000ull;                               // carry into the exponent
        double x;
        std::memcpy(&x, &bits, 8);
        ds a;
        const ds ref = ds_of_double(x);
        if (!ds_of_double_int(x, a) || a.hi != ref.hi || a.lo != ref.lo || std::signbit(a.lo) != std::signbit(ref.lo)) {
            printf("integer conversion differs: %.17g\n", x);
            return 1;
        }
    }
    {
        ds a;
        if (!ds_of_double_int(0.0, a) || a.hi != 0.0f || a.lo != 0.0f || ds_of_double_int(0x1p-71, a) ||
            ds_of_double_int(0x1p100, a)) {
            printf("integer conversion range\n");
            return 1;
        }
    }
    std::uniform_real_distribution<double> ud(0.0, 1.0);
    const long n = argc > 1 ? atol(argv[1]) : 100000;
    long nfail = 0, nbad = 0;
    double max_rel = 0.0;
    long double max_ds = 0.0L, max_fp = 0.0L;
    for (long t = 0; t < n; ++t) {
        const double R = 1.0, T = 0.05 + 8.0 * ud(rng);
        const double Uc[3] = {(ud(rng) - 0.5) * 20.0, (t % 3 == 0) ? 0.0 : ud(rng) - 0.5, 0.0};
        uint32_t w[8];
        for (int k = 0; k < 8; ++k) w[k] = static_cast<uint32_t>(rng());
        if (t % 7 == 0) w[2] = 0u;                              // u close to 0 (small -log(1 - u))
        if (t % 11 == 0) w[6] = 0xffffffffu;                    // u close to 1
        if (t % 13 == 0) { w[6] = 0u; w[7] = static_cast<uint32_t>(t) << 11; }     // tiny u
        if (t % 997 == 0) w[0] = static_cast<uint32_t>(t) & 0xffu;                 // angle near 0
        if (t % 991 == 0) w[0] = 0x40000000u + (static_cast<uint32_t>(t) & 0xffu); // near a quarter turn
        // -log(1 - u) against long double
        for (int k = 0; k < 2; ++k) {
            const uint32_t a = w[4 * k + 2], b = w[4 * k + 3];
            const ds L = ds_neg_log1m(logt, a, b);
            const long double u = static_cast<long double>(u53_host(a, b));
            const long double ex = -log1pl(-u);
            if (ex > 0) {
                const double rel = static_cast<double>(fabsl((static_cast<long double>(L.hi) + L.lo - ex) / ex));
                if (rel > max_rel) max_rel = rel;
            }
        }
        const double sq = sqrt(2.0 * R * T);
        // the cell's double-single parameters as the sampling kernels form them (integer conversions,
        // s = sqrt(2 R T) in double-single arithmetic); the conversion must equal ds_of_double
        ds U[3], s;
        const double q[5] = {1.0, Uc[0], Uc[1], Uc[2], T};
        if (!ds_maxwell_params(R, q, U, s)) {
            printf("parameters out of range at %ld\n", t);
            return 1;
        }
        for (int k = 0; k < 3; ++k) {
            const ds ref = ds_of_double(Uc[k]);
            if (U[k].hi != ref.hi || U[k].lo != ref.lo) {
                printf("integer conversion differs at %ld: %.17g\n", t, Uc[k]);
                return 1;
            }
        }
        float out[3];
        ds un[3];
        const bool ok = (t & 1) ? ds_maxwell<true>(turn, logt, U, s, w, out, un) : ds_maxwell<false>(turn, logt, U, s, w, out, un);
        // the Box-Muller pair (x: cosine, y: sine of the first angle and radius) and z (cosine of the
        // second), in double precision as the oracle evaluates it, and in long double
        const double r1 = u53_host(w[0], w[1]), r2 = 1.0 - u53_host(w[2], w[3]);
        const double r3 = u53_host(w[4], w[5]), r4 = 1.0 - u53_host(w[6], w[7]);
        const double rad = sqrt(-log(r2));
        const double fp[3] = {Uc[0] + (sq * cos(6.283185307179586 * r1)) * rad,
                              Uc[1] + (sq * sin(6.283185307179586 * r1)) * rad,
                              Uc[2] + (sq * cos(6.283185307179586 * r3)) * sqrt(-log(r4))};
        const long double kTwoPiL = 6.283185307179586476925286766559L;
        const long double La = -log1pl(-(long double)u53_host(w[2], w[3])), Lb = -log1pl(-(long double)u53_host(w[6], w[7]));
        const long double ex[3] = {(long double)Uc[0] + (long double)sq * cosl(kTwoPiL * (long double)r1) * sqrtl(La),
                                   (long double)Uc[1] + (long double)sq * sinl(kTwoPiL * (long double)r1) * sqrtl(La),
                                   (long double)Uc[2] + (long double)sq * cosl(kTwoPiL * (long double)r3) * sqrtl(Lb)};
        const long double Lk[3] = {La, La, Lb};
        for (int k = 0; k < 3; ++k) {
            // errors against the long-double evaluation with the same double inputs: of the
            // double-single value (relative to |U| + s sqrt(L)), and of the double-precision formula
            const long double S = fabsl((long double)Uc[k]) + (long double)sq * sqrtl(Lk[k]);
            if (S > 0) {
                const long double e = fabsl((long double)un[k].hi + un[k].lo - ex[k]) / S;
                if (e > max_ds) max_ds = e;
                const long double f = fabsl((long double)fp[k] - ex[k]) / S;
                if (f > max_fp) max_fp = f;
            }
        }
        if (!ok) {
            ++nfail;
            continue;
        }
        for (int k = 0; k < 3; ++k) {
            if (out[k] != static_cast<float>(fp[k])) {
                if (nbad < 5) printf("mismatch at %ld component %d: %.9g vs %.9g\n", t, k, out[k], static_cast<float>(fp[k]));
                ++nbad;
            }
        }
    }
    printf("ds-error/(|U|+s sqrt(L)) max 2^%.2f; fp64-error/(|U|+s sqrt(L)) max 2^%.2f\n", (double)log2l(max_ds), (double)log2l(max_fp));
    printf("%ld %ld %ld %.3e\n", n, nfail, nbad, max_rel);
    return nbad ? 1 : 0;
}

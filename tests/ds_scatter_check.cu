// Host-side check of the double-single scattering of single-precision records: for random pairs
// and draws, whenever ds_scatter reports success its floats must equal the single-precision
// rounding of the double-precision evaluation of the same formula (Appendix A: cos(theta) = 2 u1 - 1,
// phi = 2 pi u2, velocities (a + b)/2 +- c_r n/2), and the fallback must stay rare.
// Usage: ds_scatter_check N  -> prints the largest errors against a long-double evaluation, then
// "n fallbacks fallbacks-of-generic-cases mismatches"; exit status 1 on any mismatch.  Every 17th case draws |cos(theta)| within 2^-23 of 1, where the fallback is
// taken by design.
#include <cmath>
#include <cstdio>
#include <cstdlib>
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
    std::mt19937_64 rng(2305);
    std::normal_distribution<double> nd(0.0, 1.0);
    const long n = argc > 1 ? atol(argv[1]) : 100000;
    long nfail = 0, nfail_generic = 0, nbad = 0;
    long double max_ds = 0.0L, max_fp = 0.0L;
    for (long t = 0; t < n; ++t) {
        const float scale = (t % 7 == 0) ? 10.0f : ((t % 11 == 0) ? 0.01f : 1.0f);
        float a[3], b[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = static_cast<float>(nd(rng) * scale + (t % 5 == 0 ? 8.0 : 0.0));
            b[k] = static_cast<float>(nd(rng) * scale);
        }
        uint32_t v[4];
        for (int k = 0; k < 4; ++k) v[k] = static_cast<uint32_t>(rng());
        if (t % 13 == 0) v[2] |= 0x03ffffffu;            // angles next to the table boundaries
        if (t % 17 == 0) v[0] = (t & 1) ? 0xffffff00u : 0x000000ffu;   // |cos(theta)| close to 1
        float out[6];
        ds un[6];
        const bool ok = ds_scatter(turn, a[0], a[1], a[2], b[0], b[1], b[2], v[0], v[1], v[2], v[3], out, un);
        {
            // errors against a long-double evaluation: of the double-single values (relative to
            // c_r + |m|), and of the double-precision formula (relative to its bound)
            const long double e0 = (long double)a[0] - b[0], e1 = (long double)a[1] - b[1], e2 = (long double)a[2] - b[2];
            const long double crl = sqrtl(e0 * e0 + e1 * e1 + e2 * e2);
            const long double ctl = 2.0L * (long double)u53_host(v[0], v[1]) - 1.0L;
            const long double stl = sqrtl((1.0L - ctl) * (1.0L + ctl));
            const long double phl = 6.283185307179586476925286766559L * (long double)u53_host(v[2], v[3]);
            const long double cl[3] = {crl * stl * cosl(phl), crl * stl * sinl(phl), crl * ctl};
            const double d0 = static_cast<double>(a[0]) - b[0], d1 = static_cast<double>(a[1]) - b[1],
                         d2 = static_cast<double>(a[2]) - b[2];
            const double cr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            const double ct = 2.0 * u53_host(v[0], v[1]) - 1.0;
            const double st = sqrt(1.0 - ct * ct);
            const double ph = 6.283185307179586 * u53_host(v[2], v[3]);
            const double c[3] = {(cr * st) * cos(ph), (cr * st) * sin(ph), cr * ct};
            for (int k = 0; k < 3; ++k) {
                const long double ml = 0.5L * ((long double)a[k] + b[k]);
                const long double S = crl + fabsl(ml);
                const long double xa = ml + 0.5L * cl[k], xb = ml - 0.5L * cl[k];
                if (stl >= 0x1p-10L) {
                    const long double da = fabsl((long double)un[k].hi + un[k].lo - xa) / S;
                    const long double db = fabsl((long double)un[3 + k].hi + un[3 + k].lo - xb) / S;
                    if (da > max_ds) max_ds = da;
                    if (db > max_ds) max_ds = db;
                }
                const double m = (static_cast<double>(a[k]) + b[k]) * 0.5;
                const long double bound = 0x1p-52L * fabsl(ml) + crl * (0x1p-49L + 0x1p-52L / stl);
                const long double fa = fabsl((long double)(m + c[k] * 0.5) - xa) / bound;
                const long double fb = fabsl((long double)(m - c[k] * 0.5) - xb) / bound;
                if (fa > max_fp) max_fp = fa;
                if (fb > max_fp) max_fp = fb;
            }
        }
        if (!ok) {
            ++nfail;
            if (t % 17 != 0) ++nfail_generic;
            continue;
        }
        const double d0 = static_cast<double>(a[0]) - b[0], d1 = static_cast<double>(a[1]) - b[1],
                     d2 = static_cast<double>(a[2]) - b[2];
        const double cr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const double ct = 2.0 * u53_host(v[0], v[1]) - 1.0;
        const double st = sqrt(1.0 - ct * ct);
        const double ph = 6.283185307179586 * u53_host(v[2], v[3]);
        const double c[3] = {(cr * st) * cos(ph), (cr * st) * sin(ph), cr * ct};
        for (int k = 0; k < 3; ++k) {
            const double m = (static_cast<double>(a[k]) + b[k]) * 0.5;
            const float ra = static_cast<float>(m + c[k] * 0.5), rb = static_cast<float>(m - c[k] * 0.5);
            if (out[k] != ra || out[3 + k] != rb) {
                if (nbad < 5) printf("mismatch at %ld component %d: %.9g %.9g vs %.9g %.9g\n", t, k, out[k], out[3 + k], ra, rb);
                ++nbad;
            }
        }
    }
    printf("ds-error/(c_r+|m|) max 2^%.2f; fp64-error/bound max %.3f\n", (double)log2l(max_ds), (double)max_fp);
    printf("%ld %ld %ld %ld\n", n, nfail, nfail_generic, nbad);
    return nbad ? 1 : 0;
}

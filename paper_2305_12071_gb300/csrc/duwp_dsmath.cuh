// duwp_dsmath.cuh -- double-single (float-pair) arithmetic for the isotropic scattering of
// single-precision particle records (Appendix A), so that the post-collision velocities are
// computed on the single-precision pipes instead of the (slow) double-precision pipe.
//
// A value is an unevaluated sum hi + lo of two floats (about 48 significant bits).  Products use
// the exact product error of a fused multiply-add; sums use the exact error of a rounded sum
// (Knuth's TwoSum, Dekker's FastTwoSum); square roots take one Newton correction.  Written for
// host and device so that the arithmetic can be checked on the CPU against double precision.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace duwp {

struct ds {
    float hi, lo;
};

__host__ __device__ __forceinline__ uint32_t f_bits(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float bits_f(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}

// s + e = a + b exactly (TwoSum)
__host__ __device__ __forceinline__ ds ds_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// s + e = a + b exactly, given |a| >= |b| or a = 0 (FastTwoSum)
__host__ __device__ __forceinline__ ds ds_fast_two_sum(float a, float b)
{
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}
// p + e = a b exactly
__host__ __device__ __forceinline__ ds ds_two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
// a + b; the error is below 2^-47 of |a| + |b|
__host__ __device__ __forceinline__ ds ds_add(ds a, ds b)
{
    ds s = ds_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return ds_fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ ds ds_neg(ds a) { return {-a.hi, -a.lo}; }
// a b; relative error below 2^-46
__host__ __device__ __forceinline__ ds ds_mul(ds a, ds b)
{
    ds p = ds_two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, p.lo);
    p.lo = fmaf(a.lo, b.hi, p.lo);
    return ds_fast_two_sum(p.hi, p.lo);
}
// sqrt(a) for a > 0 (0 otherwise): y = sqrt(hi) corrected by (a - y^2) / (2 y)
__host__ __device__ __forceinline__ ds ds_sqrt(ds a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float y = sqrtf(a.hi);
    const ds y2 = ds_two_prod(y, y);
    const float r = (((a.hi - y2.hi) - y2.lo) + a.lo) / (2.0f * y);
    return ds_fast_two_sum(y, r);
}
// v 2^-frac as the nearest double (ties to even), by integer operations only: the same value as
// static_cast<double>(v) * 2^-frac for |v| < 2^63 and results in the normal range, without the
// double-precision units (few on this part).
__host__ __device__ __forceinline__ double fixed_to_double(int64_t v, int frac)
{
    if (v == 0) return 0.0;
    const uint64_t sign = v < 0 ? (1ull << 63) : 0ull;
    const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
#ifdef __CUDA_ARCH__
    const int msb = 63 - __clzll(static_cast<long long>(a));
#else
    const int msb = 63 - __builtin_clzll(a);
#endif
    int e = msb;
    uint64_t m;
    if (msb <= 52) {
        m = a << (52 - msb);
    } else {
        const int sh = msb - 52;
        const uint64_t rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        m = a >> sh;
        if (rem > half || (rem == half && (m & 1ull))) {
            m += 1ull;
            if (m == (1ull << 53)) { m >>= 1; e += 1; }
        }
    }
    const uint64_t bits = sign | (static_cast<uint64_t>(e + 1023 - frac) << 52) | (m & ((1ull << 52) - 1ull));
#ifdef __CUDA_ARCH__
    return __longlong_as_double(static_cast<long long>(bits));
#else
    double d;
    std::memcpy(&d, &bits, 8);
    return d;
#endif
}

// double-single value of a double (hi the nearest float, lo the nearest float to the rest)
__host__ __device__ __forceinline__ ds ds_of_double(double x)
{
    const float h = static_cast<float>(x);
    return {h, static_cast<float>(x - static_cast<double>(h))};
}
// double-single value of a double constant (hi the nearest float, lo the nearest float to the rest)
__host__ __device__ constexpr ds ds_const(double x)
{
    return {static_cast<float>(x), static_cast<float>(x - static_cast<double>(static_cast<float>(x)))};
}

// Whether the single-precision rounding of every value within err of v.hi + v.lo is v.hi, i.e.
// whether v.hi is the correct single-precision result even if the exact value differs from the
// computed one by up to err.  v must be normalized (|lo| at most half an ulp of hi).
__host__ __device__ __forceinline__ bool ds_rounds_to_hi(ds v, float err)
{
    const float a = fabsf(v.hi);
    if (!(a >= 1e-30f && a < 1e30f)) return false;
    const uint32_t b = f_bits(a);
    const float ulp = bits_f(b & 0x7f800000u) * 0x1p-23f;
    const float up = 0.5f * ulp;                                     // half ulp away from zero
    const float dn = (b & 0x7fffffu) ? 0.5f * ulp : 0.25f * ulp;     // toward zero (below a power of 2)
    const float l = (v.hi < 0.0f) ? -v.lo : v.lo;                    // low part in the direction of |hi|
    const float e = 1.25f * err;
    return (l + e < up) && (l - e > -dn);
}

// Double-single value of an integer |n| < 2^53 (pieces of at most 24 bits, summed; relative error below
// 2^-47).
__host__ __device__ __forceinline__ ds ds_int53(int64_t n)
{
    const uint64_t a = static_cast<uint64_t>(n < 0 ? -n : n);
    const float s = (n < 0) ? -1.0f : 1.0f;
    const float p2 = s * static_cast<float>(static_cast<uint32_t>(a >> 48)) * 0x1p48f;
    const float p1 = s * static_cast<float>(static_cast<uint32_t>((a >> 24) & 0xffffffu)) * 0x1p24f;
    const float p0 = s * static_cast<float>(static_cast<uint32_t>(a & 0xffffffu));
    return ds_add(ds_two_sum(p2, p1), {p0, 0.0f});
}

// x 2^k for a power of two f = 2^k (exact).
__host__ __device__ __forceinline__ ds ds_scale(ds x, float f) { return {x.hi * f, x.lo * f}; }

// Turn table: cos and sin of 2 pi k / 64, k = 0..63, as double-single pairs (cos hi, cos lo,
// sin hi, sin lo).
constexpr int kTurnTable = 64;

// cos and sin of phi = 2 pi u for the 53-bit uniform u = v2 2^-32 + (v3 >> 11) 2^-53: phi = 2 pi (K/64
// + r) with K = round(64 u), |r| <= 1/128 taken exactly from the bits; cos and sin of 2 pi r from
// their Taylor series (the omitted terms are below 2^-49 for |2 pi r| <= pi/64) combined with the
// turn table by the angle-addition formulas.  Absolute error below 2^-45.  ds_turn_parts gives the
// table entry (C, S) = (cos, sin)(2 pi K/64) and (cx, sx) = (cos, sin)(2 pi r).
__host__ __device__ __forceinline__ void ds_turn_parts(const float4 *turn, uint32_t v2, uint32_t v3, ds &C, ds &S,
                                                       ds &cx, ds &sx)
{
    constexpr ds kTwoPiDs = ds_const(6.283185307179586476925286766559);
    constexpr ds kMinusSixth = ds_const(-1.0 / 6.0);
    // r 2^32 = d + (v3 >> 11) 2^-21 with d = v2 - K 2^26 (32-bit wrap-around gives the sign)
    const uint32_t K = (v2 >> 26) + ((v2 >> 25) & 1u);
    const int32_t d = static_cast<int32_t>(v2 - (K << 26));
    const int32_t d_hi = d & ~3;
    const uint32_t r_lo = (static_cast<uint32_t>(d & 3) << 21) | (v3 >> 11);
    const ds r = ds_two_sum(static_cast<float>(d_hi) * 0x1p-32f, static_cast<float>(r_lo) * 0x1p-53f);
    const ds x = ds_mul(kTwoPiDs, r);                                 // |x| <= pi/64
    const ds x2 = ds_mul(x, x);
    // sin x = x + x^3 (-1/6 + x^2/120 - x^4/5040), cos x = 1 + x^2 (-1/2 + x^2/24 - x^4/720)
    const float ts = x2.hi * (1.0f / 120.0f - x2.hi * (1.0f / 5040.0f));
    sx = ds_add(x, ds_mul(ds_mul(x, x2), ds_add(kMinusSixth, {ts, 0.0f})));
    const float tc = x2.hi * (1.0f / 24.0f - x2.hi * (1.0f / 720.0f));
    cx = ds_add({1.0f, 0.0f}, ds_mul(x2, ds_two_sum(-0.5f, tc)));
    const float4 T = turn[K & (kTurnTable - 1)];
    C = {T.x, T.y};
    S = {T.z, T.w};
}

__host__ __device__ __forceinline__ void ds_turn(const float4 *turn, uint32_t v2, uint32_t v3, ds &cp, ds &sp)
{
    ds C, S, cx, sx;
    ds_turn_parts(turn, v2, v3, C, S, cx, sx);
    cp = ds_add(ds_mul(C, cx), ds_neg(ds_mul(S, sx)));
    sp = ds_add(ds_mul(S, cx), ds_mul(C, sx));
}

// cos(2 pi u) alone (same evaluation as ds_turn's cp).
__host__ __device__ __forceinline__ ds ds_turn_cos(const float4 *turn, uint32_t v2, uint32_t v3)
{
    ds C, S, cx, sx;
    ds_turn_parts(turn, v2, v3, C, S, cx, sx);
    return ds_add(ds_mul(C, cx), ds_neg(ds_mul(S, sx)));
}

// The parts of the scattering that depend only on the draw: cos(theta), sin(theta), cos(phi),
// sin(phi).  Returns false when sin(theta) < 2^-10 (the pair then takes the double-precision path).
struct DsAngles {
    ds ct, st, cp, sp;
};

__host__ __device__ __forceinline__ bool ds_scatter_angles(const float4 *turn, uint32_t v0, uint32_t v1, uint32_t v2,
                                                           uint32_t v3, DsAngles &g)
{
    // cos(theta) = 2 u1 - 1 = n 2^-52 with the integer n = m - 2^52, m = (v0 << 21) | (v1 >> 11); the
    // factors 1 - cos(theta) = (2^52 - n) 2^-52 and 1 + cos(theta) = (2^52 + n) 2^-52 are formed exactly
    // as integers, so sin(theta) carries no error amplified by 1 / sin(theta) near the poles
    const uint64_t m53 = (static_cast<uint64_t>(v0) << 21) | static_cast<uint64_t>(v1 >> 11);
    const int64_t n = static_cast<int64_t>(m53) - (1ll << 52);
    g.ct = ds_scale(ds_int53(n), 0x1p-52f);
    const ds omc = ds_int53((1ll << 52) - n), opc = ds_int53((1ll << 52) + n);
    // sin(theta) = sqrt((1 - ct)(1 + ct))
    g.st = ds_scale(ds_sqrt(ds_mul(omc, opc)), 0x1p-52f);
    if (!(g.st.hi >= 0x1p-10f)) return false;
    // phi = 2 pi u2
    ds_turn(turn, v2, v3, g.cp, g.sp);
    return true;
}

// The velocities of the pair after the collision from its angles (see ds_scatter).
__host__ __device__ __forceinline__ bool ds_scatter_apply(float au, float av, float aw, float bu, float bv, float bw,
                                                          const DsAngles &g, float out[6], ds *unrounded = nullptr)
{
    // relative speed c_r of the pair (the differences of two floats are exact pairs)
    const ds du = ds_two_sum(au, -bu), dv = ds_two_sum(av, -bv), dw = ds_two_sum(aw, -bw);
    const ds cr = ds_sqrt(ds_add(ds_add(ds_mul(du, du), ds_mul(dv, dv)), ds_mul(dw, dw)));
    // relative velocity after the collision and the two velocities (a + b)/2 +- c/2
    const ds crst = ds_mul(cr, g.st);
    const ds c[3] = {ds_mul(crst, g.cp), ds_mul(crst, g.sp), ds_mul(cr, g.ct)};
    const float a3[3] = {au, av, aw}, b3[3] = {bu, bv, bw};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const ds m = ds_two_sum(a3[k], b3[k]);
        const ds half_m = {0.5f * m.hi, 0.5f * m.lo};
        const ds half_c = {0.5f * c[k].hi, 0.5f * c[k].lo};
        const ds pa = ds_add(half_m, half_c), pb = ds_add(half_m, ds_neg(half_c));
        const float err = 0x1p-44f * (cr.hi + fabsf(half_m.hi)) + cr.hi * (0x1p-51f / g.st.hi);
        ok = ok && ds_rounds_to_hi(pa, err) && ds_rounds_to_hi(pb, err);
        out[k] = pa.hi;
        out[3 + k] = pb.hi;
        if (unrounded) {
            unrounded[k] = pa;
            unrounded[3 + k] = pb;
        }
    }
    return ok;
}

// Post-collision velocities of an accepted pair of single-precision records (isotropic VHS
// scattering, Appendix A): the relative velocity keeps its magnitude c_r and takes the direction
// with cos(theta) = 2 u1 - 1, phi = 2 pi u2, where u1 = u53(v0, v1) and u2 = u53(v2, v3) (53-bit
// uniforms u53(a, b) = a 2^-32 + (b >> 11) 2^-53).  out = (u, v, w) of A then of B, each the
// single-precision rounding of the double-precision evaluation of the same formula.  Returns false
// (out unusable) when that cannot be guaranteed: when a computed value lies within
// 2^-44 (c_r + |m|) + 2^-51 c_r / sin(theta) of a rounding boundary (m = (a+b)/2) -- the double-single
// error is below 2^-45.5 (c_r + |m|) (1 - cos and 1 + cos are formed exactly), and the
// double-precision formula deviates from the exact value by less than 2^-52 |m| + c_r (2^-49 +
// 2^-52 / sin(theta)), the last term from its sqrt(1 - cos^2) near the poles -- or when
// sin(theta) < 2^-10.  The caller then evaluates in double precision.
__host__ __device__ __forceinline__ bool ds_scatter(const float4 *turn, float au, float av, float aw, float bu,
                                                    float bv, float bw, uint32_t v0, uint32_t v1, uint32_t v2,
                                                    uint32_t v3, float out[6], ds *unrounded = nullptr)
{
    DsAngles g;
    if (!ds_scatter_angles(turn, v0, v1, v2, v3, g)) return false;
    return ds_scatter_apply(au, av, aw, bu, bv, bw, g, out, unrounded);
}

// Log table: nodes F_j = 1 + (j - kLogCenter)/256, j = 0..kLogTable-1 (covering [sqrt(1/2), 1.416]),
// entries (1/F_j hi, lo, log F_j hi, lo); entry kLogCenter is (1, 0, 0, 0).
constexpr int kLogTable = 192;
constexpr int kLogCenter = 75;

// -log(1 - u) for the 53-bit uniform u = u53(a, b) in [0, 1), relative error below 2^-46.
// 1 - u = n 2^-53 with the integer n = 2^53 - m, m = (a << 21) | (b >> 11); n = 2^e f with f in
// [0.708, 1.416), F the nearest table node (f - F formed exactly from the integers, |f - F| <= 2^-9),
// d = (f - F)/F, |d| < 2^-8.5, and
//   -log(1 - u) = (53 - e) ln 2 - log F - log(1 + d),  log(1 + d) = d - d^2/2 + d^3/3 + d^3 q(d),
// the last term (below 2^-25 |d|) in single precision.  For u near 0 the node is F = 1 and d = -u
// exactly, so small results keep their relative accuracy.
__host__ __device__ __forceinline__ ds ds_neg_log1m(const float4 *logt, uint32_t a, uint32_t b)
{
    constexpr ds kLn2 = ds_const(0.69314718055994530941723212145818);
    constexpr ds kThird = ds_const(1.0 / 3.0);
    const uint64_t m = (static_cast<uint64_t>(a) << 21) | static_cast<uint64_t>(b >> 11);
    const uint64_t n = (1ull << 53) - m;                   // 1 <= n <= 2^53
#ifdef __CUDA_ARCH__
    int e = 63 - __clzll(static_cast<long long>(n));        // n = 2^e f0, f0 in [1, 2)
#else
    int e = 63 - __builtin_clzll(n);
#endif
    const uint64_t r9 = (e >= 9) ? (n >> (e - 9)) : (n << (9 - e));    // floor(f0 512), in [512, 1023]
    int k = static_cast<int>((r9 + 1) >> 1) - 256;          // round((f0 - 1) 256), in [0, 256]
    if (k > 106) {                                          // f = f0 / 2
        e += 1;
        k = static_cast<int>(((r9 >> 1) + 1) >> 1) - 256;   // round((f - 1) 256), in [-75, 0]
    }
    // f - F = D 2^-e (e >= 8) or D 2^-8, F = (256 + k) 2^-8; |D| < 2^45
    const int64_t Fn = 256 + k;
    const int64_t D = (e >= 8) ? static_cast<int64_t>(n) - (Fn << (e - 8)) : (static_cast<int64_t>(n) << (8 - e)) - Fn;
    const float scale = bits_f(static_cast<uint32_t>(127 - (e >= 8 ? e : 8)) << 23);   // 2^-max(e, 8), e <= 54
    const float4 T = logt[k + kLogCenter];
    const ds t = ds_scale(ds_int53(D), scale);
    const ds d = ds_mul(t, {T.x, T.y});
    const ds d2 = ds_mul(d, d);
    const ds d3 = ds_mul(d2, d);
    const float df = d.hi;
    const float q = df * (-0.25f + df * (0.2f - df * (1.0f / 6.0f - df * (1.0f / 7.0f))));
    const ds lp = ds_add(d, ds_add(ds_scale(d2, -0.5f), ds_add(ds_mul(d3, kThird), {d3.hi * q, 0.0f})));
    const ds lf = ds_add({T.z, T.w}, lp);
    return ds_add(ds_mul(kLn2, {static_cast<float>(53 - e), 0.0f}), ds_neg(lf));
}

// Velocity components of a Maxwellian sample (Eq. maxsample) for single-precision records:
// xi_d = U_d + (s cos(2 pi r1)) sqrt(-log(1 - r2)), d = 0, 1, 2, with s = sqrt(2 R T), U and s as
// double-single values, (r1, r2) the 53-bit uniforms of words w[4d+2..4d+5] (w = the 14 words after
// the position's two).  out = the single-precision roundings; returns false when one of them cannot
// be guaranteed (a value within 2^-43 (|U_d| + s sqrt(-log(1 - r2))) of a rounding boundary: the
// double-single error is below 2^-44 of that, the double-precision formula's deviation below
// 2^-50), then the caller evaluates in double precision.
__host__ __device__ __forceinline__ bool ds_maxwell(const float4 *turn, const float4 *logt, const ds U[3], ds s,
                                                   const uint32_t *w, float out[3], ds *unrounded = nullptr)
{
    bool ok = true;
#pragma unroll 1   // one copy of the component code: the sampling loop is large for the instruction cache
    for (int k = 0; k < 3; ++k) {
        const ds cp = ds_turn_cos(turn, w[4 * k], w[4 * k + 1]);
        const ds L = ds_neg_log1m(logt, w[4 * k + 2], w[4 * k + 3]);
        const ds rl = ds_sqrt(L);
        const ds mag = ds_mul(s, rl);
        const ds xi = ds_add(U[k], ds_mul(mag, cp));
        const float err = 0x1p-43f * (fabsf(U[k].hi) + mag.hi);
        ok = ok && ds_rounds_to_hi(xi, err);
        out[k] = xi.hi;
        if (unrounded) unrounded[k] = xi;
    }
    return ok;
}

}  // namespace duwp

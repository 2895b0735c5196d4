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

// Double-precision bit pattern (host and device).
__host__ __device__ __forceinline__ long long dbl_bits(double x)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    long long b;
    std::memcpy(&b, &x, 8);
    return b;
#endif
}

// static_cast<float>(x) (round to nearest even) by integer operations where the result is a normal
// float, the conversion instruction otherwise (zero, subnormal results, overflow range, inf, NaN).
__host__ __device__ __forceinline__ float f32_of_double(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(dbl_bits(x));
    const int e = static_cast<int>((b >> 52) & 0x7ffu) - 1023;
    if (e < -126 || e > 127) return static_cast<float>(x);
    const uint32_t hi = static_cast<uint32_t>(b >> 32), lo = static_cast<uint32_t>(b);
    const uint32_t m23 = ((hi & 0xfffffu) << 3) | (lo >> 29), rest = lo & 0x1fffffffu;
    const uint32_t up = (rest > (1u << 28) || (rest == (1u << 28) && (m23 & 1u))) ? 1u : 0u;
    return bits_f(((hi & 0x80000000u) | (static_cast<uint32_t>(e + 127) << 23) | m23) + up);
}

// x > c for a constant c >= +0 and x < c for a constant c > 0, on the bit patterns (false for NaN x, as
// the floating-point comparison); whether x is +-0; whether x is finite
__host__ __device__ __forceinline__ bool dbl_gt(double x, double c)
{
    const long long bx = dbl_bits(x);
    return (bx & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll && bx > dbl_bits(c);
}
__host__ __device__ __forceinline__ bool dbl_lt(double x, double c)
{
    const long long bx = dbl_bits(x);
    return (bx & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll && bx < dbl_bits(c);
}
__host__ __device__ __forceinline__ bool dbl_is_zero(double x)
{
    return (static_cast<unsigned long long>(dbl_bits(x)) << 1) == 0;
}
__host__ __device__ __forceinline__ bool dbl_finite(double x)
{
    return (dbl_bits(x) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
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

// Turn table: cos and sin of 2 pi k / 128, k = 0..127, as double-single pairs (cos hi, cos lo,
// sin hi, sin lo).
constexpr int kTurnTable = 128;

// cos and sin of phi = 2 pi u for the 53-bit uniform u = v2 2^-32 + (v3 >> 11) 2^-53: phi = 2 pi (K/128
// + r) with K = round(128 u), |r| <= 1/256 taken exactly from the bits; cos and sin of x = 2 pi r from
// their Taylor series, combined with the turn table by the angle-addition formulas.  For
// |x| <= pi/128: sin x = x - x^3/6 + x^5/120 (x^7/5040 < 2^-50) and cos x = 1 - x^2/2 + x^4/24 - x^6/720
// (x^8/8! < 2^-60); x, x^2/2 and x^3/6 are carried as double-single values, the smaller terms in single
// precision (x^4/24 < 2^-26, x^5/120 < 2^-33).  Absolute error below 2^-46.  ds_turn_parts gives the
// table entry (C, S) = (cos, sin)(2 pi K/128) and (cx, sx) = (cos, sin)(2 pi r).
__host__ __device__ __forceinline__ void ds_turn_parts(const float4 *turn, uint32_t v2, uint32_t v3, ds &C, ds &S,
                                                       ds &cx, ds &sx)
{
    constexpr ds kTwoPiDs = ds_const(6.283185307179586476925286766559);
    constexpr ds kSixth = ds_const(1.0 / 6.0);
    // r 2^32 = d + (v3 >> 11) 2^-21 with d = v2 - K 2^25 (32-bit wrap-around gives the sign), |d| <= 2^24
    const uint32_t K = (v2 >> 25) + ((v2 >> 24) & 1u);
    const int32_t d = static_cast<int32_t>(v2 - (K << 25));
    const int32_t d_hi = d & ~1;
    const uint32_t r_lo = (static_cast<uint32_t>(d & 1) << 21) | (v3 >> 11);
    const ds r = ds_two_sum(static_cast<float>(d_hi) * 0x1p-32f, static_cast<float>(r_lo) * 0x1p-53f);
    const ds x = ds_mul(kTwoPiDs, r);                                 // |x| <= pi/128
    ds x2 = ds_two_prod(x.hi, x.hi);                                  // x^2 (the x.lo^2 term is below 2^-48 x^2)
    x2.lo = fmaf(2.0f * x.hi, x.lo, x2.lo);
    ds x3 = ds_two_prod(x2.hi, x.hi);                                 // x^3
    x3.lo = fmaf(x2.lo, x.hi, fmaf(x2.hi, x.lo, x3.lo));
    ds t3 = ds_two_prod(x3.hi, kSixth.hi);                            // x^3 / 6
    t3.lo = fmaf(x3.hi, kSixth.lo, fmaf(x3.lo, kSixth.hi, t3.lo));
    const float ts = (x3.hi * x2.hi) * (1.0f / 120.0f);
    const ds sa = ds_two_sum(x.hi, -t3.hi);
    sx = ds_fast_two_sum(sa.hi, ((x.lo - t3.lo) + ts) + sa.lo);
    const float tc = (x2.hi * x2.hi) * (1.0f / 24.0f - x2.hi * (1.0f / 720.0f));
    const ds ca = ds_fast_two_sum(1.0f, -0.5f * x2.hi);
    cx = ds_fast_two_sum(ca.hi, ((-0.5f * x2.lo) + tc) + ca.lo);
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

// Log table: nodes F_j = 1 + (j - kLogCenter)/1024, j = 0..kLogTable-1 (covering [0.707, 1.415]),
// entries (1/F_j hi, lo, log F_j hi, lo); entry kLogCenter is (1, 0, 0, 0).
constexpr int kLogTable = 725;
constexpr int kLogCenter = 300;

__host__ __device__ __forceinline__ int ds_clz64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __clzll(static_cast<long long>(x));
#else
    return __builtin_clzll(x);
#endif
}

// -log(1 - u) for the 53-bit uniform u = u53(a, b) in [0, 1), relative error below 2^-46.
// 1 - u = n 2^-53 with the integer n = 2^53 - m, m = (a << 21) | (b >> 11); n = 2^e f with f in
// [0.707, 1.415), F = 1 + k/1024 the nearest table node (|f - F| <= 2^-11; f - F formed exactly from
// the integers), d = (f - F)/F, |d| < 2^-10.5, and
//   -log(1 - u) = (53 - e) ln 2 - log F - log(1 + d),  log(1 + d) = d - d^2/2 + d^3/3 - d^4/4 + d^5/5
// (the omitted terms below 2^-55 |d|), with d, d^2/2 and d^3/3 as double-single values and the two
// smallest terms in single precision.  For u near 0 the node is F = 1 and d = -u exactly, so small
// results keep their relative accuracy.
__host__ __device__ __forceinline__ ds ds_neg_log1m(const float4 *logt, uint32_t a, uint32_t b)
{
    constexpr ds kLn2 = ds_const(0.69314718055994530941723212145818);
    constexpr ds kThird = ds_const(1.0 / 3.0);
    const uint64_t m = (static_cast<uint64_t>(a) << 21) | static_cast<uint64_t>(b >> 11);
    const uint64_t n = (1ull << 53) - m;                    // 1 <= n <= 2^53
    const int lz = ds_clz64(n);                              // n = 2^(63 - lz) f0, f0 in [1, 2), lz >= 10
    const uint64_t x = n << lz;                              // f0 2^63 (the low lz bits are zero)
    const uint32_t r11 = static_cast<uint32_t>(x >> 52);     // floor(f0 2048), in [2048, 4095]
    int k = static_cast<int>((r11 + 1u) >> 1) - 1024;        // round(f0 1024) - 1024, in [0, 1024]
    int h = 0;
    if (k > 424) {                                           // f = f0 / 2
        h = 1;
        k = static_cast<int>((r11 + 2u) >> 2) - 1024;        // round(f 1024) - 1024, in [-300, 0]
    }
    // f - F = D 2^-63 with F = (1024 + k)/1024: |D| <= 2^52 and the low 9 bits of D are zero, so its
    // two 32-bit halves are exact single-precision values
    const int64_t D = static_cast<int64_t>((x >> h) - (static_cast<uint64_t>(1024 + k) << 53));
    const float dh = static_cast<float>(static_cast<int32_t>(D >> 32)) * 0x1p-31f;
    const float dl = static_cast<float>(static_cast<uint32_t>(D)) * 0x1p-63f;
    const ds t = ds_two_sum(dh, dl);
    const float4 T = logt[k + kLogCenter];
    const ds d = ds_mul(t, {T.x, T.y});
    const float p = d.hi;
    ds d2 = ds_two_prod(p, p);                               // d^2
    d2.lo = fmaf(2.0f * p, d.lo, d2.lo);
    ds d3 = ds_two_prod(d2.hi, p);                           // d^3
    d3.lo = fmaf(d2.lo, p, fmaf(d2.hi, d.lo, d3.lo));
    ds t3 = ds_two_prod(d3.hi, kThird.hi);                   // d^3 / 3
    t3.lo = fmaf(d3.hi, kThird.lo, fmaf(d3.lo, kThird.hi, t3.lo));
    const float tail = (d2.hi * d2.hi) * (-0.25f + 0.2f * p);
    const ds s1 = ds_two_sum(p, -0.5f * d2.hi);
    const ds s2 = ds_fast_two_sum(s1.hi, t3.hi);
    const float lo = ((((d.lo - 0.5f * d2.lo) + t3.lo) + tail) + s1.lo) + s2.lo;
    const ds lp = ds_fast_two_sum(s2.hi, lo);                // log(1 + d)
    const float ne = static_cast<float>(lz - 10 - h);        // 53 - e, e = 63 - lz + h
    ds A = ds_two_prod(ne, kLn2.hi);
    A.lo = fmaf(ne, kLn2.lo, A.lo);
    return ds_add(ds_add(A, {-T.z, -T.w}), ds_neg(lp));
}

// {hi, lo} with hi the single-precision rounding of x and lo that of x - hi (the same pair as
// ds_of_double), by integer operations only (no double-precision unit), for x = 0 and 2^-70 <= |x| <
// 2^100; returns false outside that range (the caller then converts in double precision).
__host__ __device__ __forceinline__ bool ds_of_double_int(double x, ds &out)
{
#ifdef __CUDA_ARCH__
    const uint64_t bx = static_cast<uint64_t>(__double_as_longlong(x));
#else
    uint64_t bx;
    std::memcpy(&bx, &x, 8);
#endif
    const uint32_t hi32 = static_cast<uint32_t>(bx >> 32), lo32 = static_cast<uint32_t>(bx);
    const uint32_t sign = hi32 & 0x80000000u;
    if ((bx << 1) == 0) {
        out = {bits_f(sign), 0.0f};
        return true;
    }
    const int e = static_cast<int>((hi32 >> 20) & 0x7ffu) - 1023;    // |x| = 1.m 2^e
    if (e < -70 || e >= 100) return false;
    const uint32_t m23 = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);     // the float's 23 fraction bits
    const uint32_t rest = lo32 & 0x1fffffffu;                         // the 29 bits below them
    const uint32_t up = (rest > (1u << 28) || (rest == (1u << 28) && (m23 & 1u))) ? 1u : 0u;
    // rounding up carries into the exponent where the fraction overflows, as it should
    out.hi = bits_f((sign | (static_cast<uint32_t>(e + 127) << 23) | m23) + up);
    // |x| - |hi| = (rest - up 2^29) 2^(e-52), rounded to single precision once by the conversion
    const float r = static_cast<float>(static_cast<int32_t>(rest) - static_cast<int32_t>(up << 29)) *
                    bits_f(static_cast<uint32_t>(e - 52 + 127) << 23);
    out.lo = sign ? 0.0f - r : r;
    return true;
}

// Velocity components of a Maxwellian sample (Eq. maxsample) for single-precision records, by the
// Box-Muller transform: xi_x = U + (s cos(2 pi r1)) sqrt(-log(1 - r2)), xi_y = V + (s sin(2 pi r1))
// sqrt(-log(1 - r2)), xi_z = W + (s cos(2 pi r3)) sqrt(-log(1 - r4)), with s = sqrt(2 R T), U and s as
// double-single values, r1..r4 the 53-bit uniforms of words w[0..7] (the 8 words after the
// position's two).  out = the single-precision roundings; returns false when one of them cannot be
// guaranteed (a value within 2^-43 (|U_d| + s sqrt(-log(1 - r))) of a rounding boundary: the
// double-single error is below 2^-45 of that, the double-precision formula's deviation below
// 2^-50), then the caller evaluates in double precision.  kRolled keeps one copy of the radius code
// (for kernels whose loops crowd the instruction cache).
template <bool kRolled = true>
__host__ __device__ __forceinline__ bool ds_maxwell(const float4 *turn, const float4 *logt, const ds U[3], ds s,
                                                   const uint32_t *w, float out[3], ds *unrounded = nullptr)
{
    bool ok = true;
    auto component = [&](int k, ds mag, ds c) {
        const ds xi = ds_add(U[k], ds_mul(mag, c));
        const float err = 0x1p-43f * (fabsf(U[k].hi) + mag.hi);
        ok = ok && ds_rounds_to_hi(xi, err);
        out[k] = xi.hi;
        if (unrounded) unrounded[k] = xi;
    };
    // pair m = 0: angle w[0..1], radius w[2..3] -> x (cosine), y (sine); pair m = 1: angle w[4..5],
    // radius w[6..7] -> z (cosine)
    auto pair = [&](int m) {
        ds C, S, cx, sx;
        ds_turn_parts(turn, w[4 * m], w[4 * m + 1], C, S, cx, sx);
        const ds mag = ds_mul(s, ds_sqrt(ds_neg_log1m(logt, w[4 * m + 2], w[4 * m + 3])));
        component(2 * m, mag, ds_add(ds_mul(C, cx), ds_neg(ds_mul(S, sx))));
        if (m == 0) component(1, mag, ds_add(ds_mul(S, cx), ds_mul(C, sx)));
    };
    if (kRolled) {
#pragma unroll 1
        for (int m = 0; m < 2; ++m) pair(m);
    } else {
        pair(0);
        pair(1);
    }
    return ok;
}

// Double-single s = sqrt(2 R T) and U of a cell's Maxwellian from its double-precision state
// q = (rho, U, V, W, T) without the double-precision unit (ds_of_double_int for R, T and U; 2 R T as a
// double-single product; relative error of s below 2^-46).  Returns false where a value is outside
// the integer conversion's range.
__host__ __device__ __forceinline__ bool ds_maxwell_params(double R, const double *q, ds U[3], ds &s)
{
    ds r, t;
    bool ok = ds_of_double_int(R, r) && ds_of_double_int(q[4], t);
    for (int d = 0; d < 3; ++d) ok = ds_of_double_int(q[1 + d], U[d]) && ok;
    s = ds_sqrt(ds_mul(ds_scale(r, 2.0f), t));
    return ok;
}

}  // namespace duwp

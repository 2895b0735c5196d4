// duwp_kernels.cu -- the per-step kernels of the DUWP method (arXiv 2305.12071, Sec. 3.4) on sm_103a.
//
//   k_particles   (per cell, persistent CTAs): gather the cell's stable list (far movers, R(g-1),
//                 S(g), L(g+1)) into shared memory; absorb each particle with probability P
//                 (Eq. p); re-sample (1-P) of the wave as Maxwellian particles (Eq. maxsample);
//                 NTC/VHS collisions (Appendix A); free transport with boundaries (Step 3); write
//                 the L/S/R runs of the cell to its output block; sums of the moments that left or
//                 entered the cell (Eq. fp).
//   k_far_sort    stable order of the rare particles that moved two or more cells.
//   k_cells       (per cell): conservative update Eq. (r1), time average, primitive state, P and
//                 the slot bound of the next step.
//   k_offsets     (per cell): output block offsets of the next step (scan of the slot bounds) and
//                 the wave flux at every interface.
#include <cstdio>

#include "duwp_launch.h"

namespace duwp {

__device__ __forceinline__ void set_err(int32_t *err, int code) { atomicCAS(err, 0, code); }

// ------------------------------------------------------------------------------------------
// Record access (FP32 records are one 16-byte vector; FP64 records two).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ RecF ld_rec(const RecF *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return RecF{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ RecD ld_rec(const RecD *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return RecD{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st_rec(RecF *p, const RecF &r)
{
    *reinterpret_cast<float4 *>(p) = make_float4(r.xl, r.u, r.v, r.w);
}
__device__ __forceinline__ void st_rec(RecD *p, const RecD &r)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(r.xl, r.u);
    reinterpret_cast<double2 *>(p)[1] = make_double2(r.v, r.w);
}

// Storage rounding of a value computed in FP64.
__device__ __forceinline__ float store_val(double x, float) { return __double2float_rn(x); }
__device__ __forceinline__ double store_val(double x, double) { return x; }

// ------------------------------------------------------------------------------------------
// Free transport in cell units with the boundary conditions (Step 3).  The position update
// x + xi dt/dx is one fused multiply-add in the record precision; the new cell is its floor.
// Returns the new local cell or -1 (the particle left the domain).
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int64_t apply_walls(const InstDev &I, int64_t dest, T &x, T &u, bool &refl)
{
    const int64_t C = I.C;
    for (int it = 0; it < 64; ++it) {
        if (dest < 0) {
            if (I.bc_left == 1) {
                dest = -dest - 1;
                x = T(1) - x;
                if (x >= T(1)) { x = T(0); dest += 1; }
                u = -u;
                refl = !refl;
                continue;
            }
            if (I.bc_left == 2) { dest = ((dest % C) + C) % C; continue; }
            return -1;
        }
        if (dest >= C) {
            if (I.bc_right == 1) {
                dest = 2 * C - dest - 1;
                x = T(1) - x;
                if (x >= T(1)) { x = T(0); dest += 1; }
                u = -u;
                refl = !refl;
                continue;
            }
            if (I.bc_right == 2) { dest = dest % C; continue; }
            return -1;
        }
        return dest;
    }
    return -1;   // more than 64 wall reflections within one step: removed
}

__device__ __forceinline__ int64_t transport(const InstDev &I, int64_t cell, float &xl, float &u, bool &refl)
{
    const float s = __fmaf_rn(u, I.dtdx_f, xl);
    if (!(fabsf(s) < 1e15f)) return -1;
    const float fk = floorf(s);
    float x = __fsub_rn(s, fk);
    // the integral value fk converts exactly; a 32-bit conversion covers every displacement
    // below 2^30 cells (the 64-bit one is reserved for larger ones)
    int64_t k = (fabsf(fk) < 1073741824.0f) ? static_cast<int64_t>(__float2int_rz(fk)) : static_cast<int64_t>(fk);
    if (x >= 1.0f) { x = 0.0f; k += 1; }
    xl = x;
    return apply_walls<float>(I, cell + k, xl, u, refl);
}

__device__ __forceinline__ int64_t transport(const InstDev &I, int64_t cell, double &xl, double &u, bool &refl)
{
    const double s = __fma_rn(u, I.dtdx, xl);
    if (!(fabs(s) < 1e15)) return -1;
    const double fk = floor(s);
    double x = __dsub_rn(s, fk);
    int64_t k = static_cast<int64_t>(fk);
    if (x >= 1.0) { x = 0.0; k += 1; }
    xl = x;
    return apply_walls<double>(I, cell + k, xl, u, refl);
}

// ------------------------------------------------------------------------------------------
// Maxwellian sample at the primitive state q (Eq. maxsample): per component
// xi = U + sqrt(2RT) cos(2 pi r1) sqrt(-ln r2), r2 in (0,1]; position uniform in the cell.
// Particle j of a cell uses counters (id, 4j..4j+3, step, SAMPLE): uniforms 0 -> position,
// (1,2) -> x, (3,4) -> y, (5,6) -> z.
// ------------------------------------------------------------------------------------------
template <typename Rec>
__device__ __noinline__ Rec sample_particle(const InstDev &I, uint32_t id, uint32_t j, uint32_t step, const double *q)
{
    uint32_t w[16];
#pragma unroll
    for (uint32_t t = 0; t < 4; ++t) draw(I, id, 4u * j + t, step, kSample, w + 4 * t);
    double un[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) un[k] = u53(w[2 * k], w[2 * k + 1]);
    const double sq = sqrt(2.0 * I.R * q[4]);
    double xi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double r1 = un[1 + 2 * d];
        const double r2 = 1.0 - un[2 + 2 * d];
        xi[d] = q[1 + d] + (sq * cos(kTwoPi * r1)) * sqrt(-log(r2));
    }
    Rec r;
    using T = decltype(r.xl);
    T x = store_val(un[0], T());
    if (x >= T(1)) x = sizeof(T) == 4 ? T(0x1.fffffep-1f) : T(un[0]);
    r.xl = x;
    r.u = store_val(xi[0], T());
    r.v = store_val(xi[1], T());
    r.w = store_val(xi[2], T());
    return r;
}

// ------------------------------------------------------------------------------------------
// Block-wide helpers
// ------------------------------------------------------------------------------------------

// Exclusive scan of a 64-bit value over the CTA (in thread order); total returned via *tot.
__device__ __forceinline__ uint64_t block_scan_u64(uint64_t v, uint64_t *s_w, uint64_t *tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t t = (lane < nw) ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) s_w[lane] = t;
    }
    __syncthreads();
    const uint64_t pre = (warp > 0) ? s_w[warp - 1] : 0;
    *tot = s_w[nw - 1];
    __syncthreads();
    return pre + x - v;
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Lower bound of `key` in the far list ordered by (dest, src, q): first index with (dest, src) >= key.
template <typename Rec>
__device__ int far_lower(const FarItem<Rec> *f, int n, int dest, int src)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const bool less = (f[mid].dest < dest) || (f[mid].dest == dest && f[mid].src < src);
        if (less) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------------------------------
// NTC collisions of one cell (Appendix A), one warp.  Candidates are taken in order in batches of
// up to 32: the batch is cut before the first candidate that shares a particle with an earlier
// one in the batch, and after the first whose c_r raises c_max; inside such a prefix the
// candidates touch disjoint particles and see the same c_max, so doing them at once gives exactly
// the sequential result.  The acceptance test (c_r/c_max)^{1-2 upsilon} > u is first decided in
// FP32 with a margin far above its error; only draws within the margin take the FP64 pow.
// ------------------------------------------------------------------------------------------
// Majorant factor (c_max/c_ref)^{-2 upsilon} of the NTC count; kept per cell and recomputed only when
// c_max is raised.
__device__ inline double majorant_factor(const InstDev &I, double cmax)
{
    return (I.upsilon == 0.0) ? 1.0 : pow(cmax / I.c_ref, -2.0 * I.upsilon);
}

// NTC candidate count of a cell with N particles (Appendix A, nondimensional form), rounded with the
// cell's ROUND draw 1; -1 when the count is absurd (over 1e8).  The density ratio uses the
// precomputed m_p/(dx rho_ref) and the majorant factor comes from the per-cell cache, so the product
// may differ from the plain left-to-right evaluation by a few ulps; the rounded count differs only
// when N_sel + u lies within those ulps of an integer.
__device__ inline int64_t ntc_candidates(const InstDev &I, uint32_t id, uint32_t step, int N, double rho_t, double cmax,
                                         double fmaj)
{
    if (N < 2) return 0;
    const double rr = (I.ntc_rate == 1) ? rho_t * I.inv_rho_ref : static_cast<double>(N) * I.ntc_rr;
    const double nsel = I.ntc_A * rr * (static_cast<double>(N) - 1.0) * fmaj * cmax;
    if (!(nsel < 1e8)) return -1;
    uint32_t w[4];
    draw(I, id, 1u, step, kRound, w);
    return static_cast<int64_t>(floor(nsel + u53(w[0], w[1])));
}

// Relative speed of two records, single precision (relative error below 1e-6).
__device__ __forceinline__ float rel_speed_f32(const RecF &A, const RecF &B)
{
    const float d0 = A.u - B.u, d1 = A.v - B.v, d2 = A.w - B.w;
    return sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
}
__device__ __forceinline__ float rel_speed_f32(const RecD &A, const RecD &B)
{
    const float d0 = static_cast<float>(A.u - B.u), d1 = static_cast<float>(A.v - B.v), d2 = static_cast<float>(A.w - B.w);
    return sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
}
template <typename Rec>
__device__ __forceinline__ double rel_speed(const Rec &A, const Rec &B)
{
    const double d0 = static_cast<double>(A.u) - static_cast<double>(B.u);
    const double d1 = static_cast<double>(A.v) - static_cast<double>(B.v);
    const double d2 = static_cast<double>(A.w) - static_cast<double>(B.w);
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

// The nc candidates of a cell in order (nc from ntc_candidates).  tidx (optional): sorted list
// indices of the records held in `list` (the touched particles); without it `list` is the whole
// cell list.  Both the test c_r > c_max and the acceptance u < (c_r/c_max)^{1-2 upsilon} are first
// decided in single precision with margins far above its error; exact double-precision values are
// computed for draws inside the margins and for every accepted pair (its scattering).
template <typename Rec>
__device__ __noinline__ void collide_warp(const InstDev &I, uint32_t id, uint32_t step, Rec *list, int N, int64_t nc,
                                          double &cmax, int &nacc, int *s_ab, const int *tidx, int ntouch)
{
    using T = decltype(list[0].xl);
    const int lane = threadIdx.x & 31;
    nacc = 0;
    if (N < 2 || nc <= 0) return;
    uint32_t w[4];
    const double expo = 1.0 - 2.0 * I.upsilon;
    const float expo_f = static_cast<float>(expo);
    int acc = 0;
    double cm = cmax;
    for (int64_t k0 = 0; k0 < nc;) {
        const int64_t k = k0 + lane;
        const bool act = k < nc;
        uint32_t a = 0, b = 0;
        double ua = 0.0;
        if (act) {
            draw(I, id, static_cast<uint32_t>(2 * k), step, kCollide, w);
            a = idx32(w[0], static_cast<uint32_t>(N));
            b = idx32(w[1], static_cast<uint32_t>(N - 1));
            if (b >= a) ++b;
            ua = u53(w[2], w[3]);
        }
        s_ab[lane] = act ? static_cast<int>(a) : -1;
        s_ab[32 + lane] = act ? static_cast<int>(b) : -2;
        __syncwarp();
        bool conf = false;
        for (int j = 0; j < lane; ++j) {
            const int aj = s_ab[j], bj = s_ab[32 + j];
            conf |= (static_cast<int>(a) == aj) | (static_cast<int>(a) == bj) | (static_cast<int>(b) == aj) |
                    (static_cast<int>(b) == bj);
        }
        const unsigned cmask = __ballot_sync(0xffffffffu, act && conf);
        const int navail = static_cast<int>(min(static_cast<int64_t>(32), nc - k0));
        const int m1 = cmask ? min(navail, __ffs(cmask) - 1) : navail;
        Rec A, B;
        float cr32 = 0.f;
        double cr = 0.0;
        bool exact = false;
        uint32_t sa = a, sb = b;
        if (tidx && lane < m1) {
            int lo = 0, hi = ntouch;
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (tidx[mid] < static_cast<int>(a)) lo = mid + 1; else hi = mid; }
            sa = static_cast<uint32_t>(lo);
            lo = 0; hi = ntouch;
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (tidx[mid] < static_cast<int>(b)) lo = mid + 1; else hi = mid; }
            sb = static_cast<uint32_t>(lo);
        }
        const float cm32 = static_cast<float>(cm);
        if (lane < m1) {
            A = list[sa];
            B = list[sb];
            cr32 = rel_speed_f32(A, B);
            if (cr32 > cm32 * 0.99999f) {      // possibly above c_max: decide exactly
                cr = rel_speed(A, B);
                exact = true;
            }
        }
        const unsigned rmask = __ballot_sync(0xffffffffu, lane < m1 && exact && cr > cm);
        const int fr = rmask ? __ffs(rmask) - 1 : 32;
        const int m = min(m1, fr + 1);
        const double cr_r = __shfl_sync(0xffffffffu, cr, fr < 32 ? fr : 0);
        bool accd = false;
        if (lane < m) {
            if (lane == fr) {
                accd = true;                    // c_max = c_r: acceptance probability 1
            } else if (expo == 0.0) {
                accd = ua < 1.0;
            } else {
                const float x32 = cr32 / cm32;
                const float p32 = (I.upsilon == 0.0) ? x32 : exp2f(expo_f * log2f(x32));
                const double p = static_cast<double>(p32);
                const double margin = 1e-4 * p + 1e-7;
                if (ua < p - margin) accd = true;
                else if (ua > p + margin) accd = false;
                else {
                    if (!exact) { cr = rel_speed(A, B); exact = true; }
                    const double x = cr / cm;
                    accd = ua < ((I.upsilon == 0.0) ? x : pow(x, expo));
                }
            }
            if (accd) {
                if (!exact) cr = rel_speed(A, B);
                uint32_t v[4];
                draw(I, id, static_cast<uint32_t>(2 * k + 1), step, kCollide, v);
                const double ct = 2.0 * u53(v[0], v[1]) - 1.0;
                const double st = sqrt(1.0 - ct * ct);
                double sp, cp;
                sincos(kTwoPi * u53(v[2], v[3]), &sp, &cp);
                const double c0 = (cr * st) * cp, c1 = (cr * st) * sp, c2 = cr * ct;
                const double au = A.u, av = A.v, aw = A.w, bu = B.u, bv = B.v, bw = B.w;
                const double m0 = (au + bu) * 0.5, mm1 = (av + bv) * 0.5, m2 = (aw + bw) * 0.5;
                A.u = store_val(m0 + c0 * 0.5, T());
                A.v = store_val(mm1 + c1 * 0.5, T());
                A.w = store_val(m2 + c2 * 0.5, T());
                B.u = store_val(m0 - c0 * 0.5, T());
                B.v = store_val(mm1 - c1 * 0.5, T());
                B.w = store_val(m2 - c2 * 0.5, T());
                list[sa] = A;
                list[sb] = B;
            }
        }
        acc += __popc(__ballot_sync(0xffffffffu, accd));
        if (fr < m) cm = cr_r;
        __syncwarp();
        k0 += m;
    }
    cmax = cm;
    nacc = acc;
}

// ------------------------------------------------------------------------------------------
// Exact fixed-point sums of particle moments: velocities at 2^-40, |xi|^2/2 at 2^-32.  Integer
// sums do not depend on the order of accumulation, so the per-cell flux sums are identical for
// every launch shape, and the global particle-flux ledger telescopes exactly.
// ------------------------------------------------------------------------------------------
// x * 2^S rounded to the nearest integer (halves away from zero), from the bits of the float with
// integer arithmetic only; |x| must stay below 2^(62-S) (guarded by the caller's range check).
template <int S>
__device__ __forceinline__ long long fx_bits(float x)
{
    const unsigned bits = __float_as_uint(x);
    const unsigned be = (bits >> 23) & 0xffu;
    const unsigned long long mant = (bits & 0x7fffffu) | (be ? 0x800000u : 0u);
    const int e = static_cast<int>(be ? be : 1u) - 150 + S;   // |x| 2^S = mant 2^e
    long long v;
    if (e >= 0) v = static_cast<long long>(mant << e);
    else if (e > -32) v = static_cast<long long>((mant + (1ull << (-e - 1))) >> (-e));
    else v = 0;
    return (bits >> 31) ? -v : v;
}
__device__ __forceinline__ long long fx_vel(float x) { return fx_bits<40>(x); }
__device__ __forceinline__ long long fx_vel(double x) { return __double2ll_rn(x * 1099511627776.0); }
// largest velocity component accepted in the exact sums (2^14; |xi|^2 then stays below 2^30):
// faster particles are reported as overflow
__device__ __forceinline__ bool fx_in_range(float x) { return fabsf(x) < 16384.0f; }
__device__ __forceinline__ bool fx_in_range(double x) { return fabs(x) < 16384.0; }

// |xi|^2/2 * 2^32: squares split exactly into float pairs (TwoProd by fma), summed error-free.
__device__ __forceinline__ long long fx_energy(float u, float v, float w)
{
    const float pu = u * u, pv = v * v, pw = w * w;
    const float qu = __fmaf_rn(u, u, -pu), qv = __fmaf_rn(v, v, -pv), qw = __fmaf_rn(w, w, -pw);
    float s = pu + pv;
    float bb = s - pu;
    float e = (pu - (s - bb)) + (pv - bb);
    const float s2 = s + pw;
    bb = s2 - s;
    e += (s - (s2 - bb)) + (pw - bb);
    const float lo = ((qu + qv) + qw) + e;
    return fx_bits<31>(s2) + fx_bits<31>(lo);
}
__device__ __forceinline__ long long fx_energy(double u, double v, double w)
{
    return __double2ll_rn((u * u + v * v + w * w) * 2147483648.0);
}

// ------------------------------------------------------------------------------------------
// Particle kernel: one warp per cell, no block-wide barriers.
//
// Output block of a cell s (2 x slots records, slots = the bound on its list after re-sampling):
// particles that stay (S) are written forward from the block start, those moving one cell left
// (L) forward from the middle, those moving one cell right (R) backward from the end; each run
// keeps the order the particles had before transport.  The sorted list of cell g for the next
// step reads R(g-1) from its end backwards, then S(g), then L(g+1).
//
// Two ways through a cell:
//   direct  (P = 0 and at most 32 NTC candidates): the candidate pairs are drawn first (they depend
//           only on counters), the touched particles are copied to shared memory and collided
//           there, then one streaming pass reads the arrived runs (and samples the re-sampled
//           particles), substitutes the touched ones, transports and writes;
//   staged  (P > 0, or more candidates): survivors of the absorption draw and the re-sampled
//           particles are written to the first half of the cell's own output block, collided
//           there, then streamed from there (stayers are written back in place, never ahead of
//           the read position).
// ------------------------------------------------------------------------------------------
constexpr int kTouchCap = 64;
constexpr int kMaxCand = 32;

template <typename Rec>
struct WarpShared {
    int b, i, ghost, skip, staged;
    int n_in, n_surv, n_new, n_tot, slots;
    int nfb, fb, Rn, Sn, Ln, nfa, fa;
    long long Rend, Sa, La, off_out;
    double P, rho_t, cmax;
    double q[5];
    int valid, ncand, nacc, ntouch;
    int nL, nS, nR;
    int ab[64];
    int tidx[kTouchCap];
    Rec trec[kTouchCap];
    long long acc[4][32];    // lane-private fixed-point sums of the rare cases (u, v, w, e)
};

// Record of position k of the cell's arrived (sorted) list.
template <typename Rec>
__device__ __forceinline__ Rec fetch_arrived(int k, int nfb, int fb, int Rn, long long Rend, int Sn, long long Sa,
                                             int Ln, long long La, int fa, const Rec *in, const FarItem<Rec> *fs)
{
    int r = k;
    if (r < nfb) return fs[fb + r].rec;
    r -= nfb;
    if (r < Rn) return ld_rec(in + (Rend - 1 - r));
    r -= Rn;
    if (r < Sn) return ld_rec(in + (Sa + r));
    r -= Sn;
    if (r < Ln) return ld_rec(in + (La + r));
    r -= Ln;
    return fs[fa + r].rec;
}

// Plain (coherent) loads for records written earlier in the same kernel.
__device__ __forceinline__ RecF ld_rec_rw(const RecF *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return RecF{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ RecD ld_rec_rw(const RecD *p)
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    return RecD{a.x, a.y, b.x, b.y};
}

template <typename Rec>
__device__ __forceinline__ int touched_slot(const WarpShared<Rec> &S, int x)
{
    int lo = 0, hi = S.ntouch;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (S.tidx[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Header of cell g (lane 0).
template <typename Rec>
__device__ __noinline__ void cell_header(const EngineDev &E, int rp, int g, WarpShared<Rec> &S)
{
    const int wp = 1 - rp;
    S.skip = 0;
    S.staged = 0;
    S.ncand = S.nacc = 0;
    S.nL = S.nS = S.nR = 0;
    S.n_in = S.n_surv = S.n_new = S.n_tot = 0;
    S.nfb = S.nfa = S.fb = S.fa = 0;
    S.Rn = S.Sn = S.Ln = 0;
    S.ntouch = 0;
    S.b = E.cell_inst[g];
    if (S.b < 0) { S.skip = 1; return; }
    const InstDev &I = E.inst[S.b];
    S.i = g - I.cell_base - 1;
    S.ghost = (S.i < 0) ? 1 : (S.i >= I.C ? 2 : 0);
    S.slots = E.slots[g];
    S.off_out = E.off[wp][g];
    if (S.off_out + 2 * static_cast<long long>(S.slots) > E.capacity) {
        set_err(E.err, kErrOverflow);
        S.skip = 1;
        return;
    }
    const uint32_t step = I.step;
    if (S.ghost) {
        const int side = S.ghost - 1;
        const int bc = side ? I.bc_right : I.bc_left;
        if (bc != 0) { S.skip = 1; return; }
        double q[5];
        const bool ok = ghost_prim(I, side, q, false, q);
        for (int k = 0; k < 5; ++k) S.q[k] = q[k];
        S.valid = ok;
        S.P = split_fraction(I, q, ok);
        S.rho_t = 0.0;
        S.cmax = 0.0;
        S.n_new = ok ? static_cast<int>(resample_count(I, static_cast<uint32_t>(S.i + 1), step, S.P, q[0])) : 0;
        S.n_tot = S.n_new;
        if (S.n_tot > S.slots) { set_err(E.err, kErrOverflow); S.skip = 1; }
        return;
    }
    for (int k = 0; k < 5; ++k) S.q[k] = E.prim[5 * g + k];
    S.valid = E.valid[g];
    S.P = E.P[g];
    S.rho_t = E.psi[5 * g];
    S.cmax = E.cmax[g];
    S.Rend = E.off[rp][g - 1] + 2 * static_cast<long long>(E.slotsb[rp][g - 1]);
    S.Rn = E.nR[rp][g - 1];
    S.Sa = E.off[rp][g];
    S.Sn = E.nS[rp][g];
    S.La = E.off[rp][g + 1] + E.slotsb[rp][g + 1];
    S.Ln = E.nL[rp][g + 1];
    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
    const int nf = E.far_count[1];
    if (nf > 0) {
        const int lo = far_lower(fs, nf, g, INT32_MIN);
        const int mid = far_lower(fs, nf, g, g + 2);
        const int hi = far_lower(fs, nf, g + 1, INT32_MIN);
        S.fb = lo;
        S.nfb = mid - lo;
        S.fa = mid;
        S.nfa = hi - mid;
    }
    S.n_in = S.nfb + S.Rn + S.Sn + S.Ln + S.nfa;
    if (S.n_in != E.cnt[g] || S.n_in > S.slots) {
        set_err(E.err, kErrOverflow);
        S.skip = 1;
        return;
    }
    if (S.P > 0.0) { S.staged = 1; return; }
    // P = 0: nothing is absorbed; the re-sampled count and the NTC candidate count are known now
    const uint32_t id = static_cast<uint32_t>(S.i + 1);
    S.n_surv = S.n_in;
    const double rho_w = S.rho_t - static_cast<double>(S.n_in) * I.mp_over_dx;
    S.n_new = S.valid ? static_cast<int>(resample_count(I, id, step, 0.0, rho_w)) : 0;
    S.n_tot = S.n_in + S.n_new;
    if (S.n_tot > S.slots) { set_err(E.err, kErrOverflow); S.skip = 1; return; }
    const int64_t nc = ntc_candidates(I, id, step, S.n_tot, S.rho_t, S.cmax, E.fmaj[g]);
    if (nc < 0) { set_err(E.err, kErrOverflow); S.skip = 1; return; }
    S.ncand = static_cast<int>(nc);
    if (nc > kMaxCand) S.staged = 1;
}

struct StreamState {
    long long pS, pL, pR;                 // next write position of the S, L (forward) and R (backward) runs
    long long *acc;                       // this lane's column of the warp's rare-path sums (stride 32)
    int ngone = 0;                        // far movers and removed particles of this lane
    bool range_ok = true;
};

struct StreamCtx {
    const InstDev *I;
    const EngineDev *E;
    int ci, cell_base, g;
};

// One group of 32 consecutive list positions (lanes in list order): transport, classification and
// stable writes to the three runs.  The moments of the L and R runs are summed afterwards from the
// runs themselves; only the rare cases are summed here: particles that move two or more cells or
// leave the domain (their pre-transport moments leave the cell), and wall reflections (the normal
// momentum a reflected particle carries changes sign: +2 u after the reflection).
template <typename Rec>
__device__ __forceinline__ void stream_group(const StreamCtx &cx, Rec v, bool valid, int k, Rec *out,
                                             FarItem<Rec> *fa, StreamState &st)
{
    using T = decltype(Rec().xl);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int c = 5;
    if (valid) {
        const T u0 = v.u;
        T xl = v.xl, uu = v.u;
        bool refl = false;
        const int64_t d = transport(*cx.I, cx.ci, xl, uu, refl);
        v.xl = xl;
        v.u = uu;
        if (d < 0) c = 4;
        else if (d == cx.ci - 1) c = 0;
        else if (d == cx.ci) c = 1;
        else if (d == cx.ci + 1) c = 2;
        else c = 3;
        if (refl || c >= 3) {
            long long *a = st.acc;
            st.range_ok = st.range_ok && fx_in_range(u0) && fx_in_range(v.v) && fx_in_range(v.w);
            if (c >= 3) {
                ++st.ngone;
                a[0] -= fx_vel(u0);
                a[32] -= fx_vel(v.v);
                a[64] -= fx_vel(v.w);
                a[96] -= fx_energy(u0, v.v, v.w);
            } else {
                a[0] += fx_vel(uu) - fx_vel(u0);
            }
            if (c == 3) {
                const EngineDev &E = *cx.E;
                const int slot = atomicAdd(&E.far_count[0], 1);
                if (slot < E.far_cap) {
                    FarItem<Rec> it;
                    it.dest = cx.cell_base + 1 + static_cast<int>(d);
                    it.src = cx.g;
                    it.q = k;
                    it.pad = 0;
                    it.rec = v;
                    fa[slot] = it;
                } else {
                    set_err(E.err, kErrOverflow);
                }
            }
        }
    }
    const unsigned mL = __ballot_sync(0xffffffffu, c == 0);
    const unsigned mS = __ballot_sync(0xffffffffu, c == 1);
    const unsigned mR = __ballot_sync(0xffffffffu, c == 2);
    if (c == 1) st_rec(out + st.pS + __popc(mS & lt), v);
    else if (c == 0) st_rec(out + st.pL + __popc(mL & lt), v);
    else if (c == 2) st_rec(out + st.pR - __popc(mR & lt), v);
    st.pS += __popc(mS);
    st.pL += __popc(mL);
    st.pR -= __popc(mR);
}

// Fixed-point sums (u, v, w, |xi|^2/2) of n contiguous records, each lane a strided share.
template <typename Rec>
__device__ __forceinline__ void run_sums(const Rec *p, int n, long long s[4], bool &ok)
{
    for (int j = threadIdx.x & 31; j < n; j += 32) {
        const Rec v = ld_rec_rw(p + j);
        ok = ok && fx_in_range(v.u) && fx_in_range(v.v) && fx_in_range(v.w);
        s[0] += fx_vel(v.u);
        s[1] += fx_vel(v.v);
        s[2] += fx_vel(v.w);
        s[3] += fx_energy(v.u, v.v, v.w);
    }
}

template <typename Rec, int kMinBlocks>
__global__ void __launch_bounds__(kMinBlocks == 1 ? 512 : 128, kMinBlocks) k_particles(EngineDev E, int rp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    WarpShared<Rec> &S = reinterpret_cast<WarpShared<Rec> *>(smraw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int wp = 1 - rp;
    const Rec *in = static_cast<const Rec *>(E.buf[rp]);
    Rec *out = static_cast<Rec *>(E.buf[wp]);
    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
    FarItem<Rec> *fa = static_cast<FarItem<Rec> *>(E.far_app);

    for (;;) {
        int g = 0;
        if (lane == 0) g = atomicAdd(E.ticket, 1);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= E.G) break;
        if (lane == 0) cell_header<Rec>(E, rp, g, S);
        __syncwarp();
        if (!S.skip) {
            const InstDev &I = E.inst[S.b];
            const uint32_t step = I.step;
            const uint32_t id = static_cast<uint32_t>(S.i + 1);
            const int ci = S.i, cell_base = I.cell_base;
            const int nfb = S.nfb, fb = S.fb, Rn = S.Rn, Sn = S.Sn, Ln = S.Ln, fa_ = S.fa;
            const long long Rend = S.Rend, Sa = S.Sa, La = S.La, off = S.off_out;
            const int slots = S.slots;
            const int n_in = S.n_in;
            Rec *stage = out + off;
            bool ok = true;

            if (S.staged) {
                // ---- survivors of the absorption draw (Eq. p) into the first half, in order
                const double P = S.P;
                int run = 0;
                for (int base = 0; base < n_in; base += 32) {
                    const int k = base + lane;
                    Rec v;
                    bool keep = false;
                    if (k < n_in) {
                        v = fetch_arrived<Rec>(k, nfb, fb, Rn, Rend, Sn, Sa, Ln, La, fa_, in, fs);
                        keep = true;
                        if (P > 0.0) {
                            uint32_t w[4];
                            draw(I, id, static_cast<uint32_t>(k), step, kAbsorb, w);
                            keep = !(u53(w[0], w[1]) < P);
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (keep) st_rec(stage + run + __popc(m & lt), v);
                    run += __popc(m);
                }
                if (lane == 0) {
                    S.n_surv = run;
                    const double rho_w = S.rho_t - static_cast<double>(run) * I.mp_over_dx;
                    S.n_new = S.valid ? static_cast<int>(resample_count(I, id, step, P, rho_w)) : 0;
                    S.n_tot = run + S.n_new;
                    if (S.n_tot > slots) { set_err(E.err, kErrOverflow); S.skip = 1; }
                }
                __syncwarp();
                if (S.skip) {
                    ok = false;
                } else {
                    // ---- re-sampled particles (Eq. maxsample) after the survivors, then collisions
                    const int n_surv = S.n_surv;
                    for (int j = lane; j < S.n_new; j += 32)
                        st_rec(stage + n_surv + j, sample_particle<Rec>(I, id, static_cast<uint32_t>(j), step, S.q));
                    __syncwarp();
                    double cmax = S.cmax;
                    int na = 0;
                    int64_t nc = ntc_candidates(I, id, step, S.n_tot, S.rho_t, cmax, E.fmaj[g]);
                    if (nc < 0) {
                        if (lane == 0) set_err(E.err, kErrOverflow);
                        nc = 0;
                    }
                    collide_warp<Rec>(I, id, step, stage, S.n_tot, nc, cmax, na, S.ab, nullptr, 0);
                    if (lane == 0) {
                        S.ncand = static_cast<int>(nc);
                        S.nacc = na;
                        if (cmax != S.cmax) {
                            E.cmax[g] = cmax;
                            E.fmaj[g] = majorant_factor(I, cmax);
                        }
                    }
                    __syncwarp();
                }
            } else if (S.ncand > 0) {
                // ---- direct way: stage only the particles the candidates touch
                const int nc = S.ncand, N = S.n_tot;
                int a = 0x7fffffff, b = 0x7fffffff;
                if (lane < nc) {
                    uint32_t w[4];
                    draw(I, id, static_cast<uint32_t>(2 * lane), step, kCollide, w);
                    a = static_cast<int>(idx32(w[0], static_cast<uint32_t>(N)));
                    b = static_cast<int>(idx32(w[1], static_cast<uint32_t>(N - 1)));
                    if (b >= a) ++b;
                }
                S.ab[lane] = a;
                S.ab[32 + lane] = b;
                __syncwarp();
                // rank sort of the 64 picks, then drop repeats
                int ra = 0, rb = 0;
                for (int j = 0; j < 64; ++j) {
                    const int x = S.ab[j];
                    ra += (x < a) || (x == a && j < lane);
                    rb += (x < b) || (x == b && j < 32 + lane);
                }
                __syncwarp();
                S.tidx[ra] = a;
                S.tidx[rb] = b;
                __syncwarp();
                const int v0 = S.tidx[2 * lane], v1 = S.tidx[2 * lane + 1];
                const int p0 = (2 * lane == 0) ? 0x7ffffffe : S.tidx[2 * lane - 1];
                const bool k0 = v0 != 0x7fffffff && v0 != p0;
                const bool k1 = v1 != 0x7fffffff && v1 != v0;
                const unsigned m0 = __ballot_sync(0xffffffffu, k0), m1 = __ballot_sync(0xffffffffu, k1);
                const int before = __popc(m0 & lt) + __popc(m1 & lt);
                __syncwarp();
                if (k0) S.tidx[before] = v0;
                if (k1) S.tidx[before + (k0 ? 1 : 0)] = v1;
                const int nt = __popc(m0) + __popc(m1);
                if (lane == 0) S.ntouch = nt;
                __syncwarp();
                for (int t = lane; t < nt; t += 32) {
                    const int x = S.tidx[t];
                    S.trec[t] = (x < n_in) ? fetch_arrived<Rec>(x, nfb, fb, Rn, Rend, Sn, Sa, Ln, La, fa_, in, fs)
                                           : sample_particle<Rec>(I, id, static_cast<uint32_t>(x - n_in), step, S.q);
                }
                __syncwarp();
                double cmax = S.cmax;
                int na = 0;
                collide_warp<Rec>(I, id, step, S.trec, N, nc, cmax, na, S.ab, S.tidx, nt);
                if (lane == 0) {
                    S.nacc = na;
                    if (cmax != S.cmax) {
                        E.cmax[g] = cmax;
                        E.fmaj[g] = majorant_factor(I, cmax);
                    }
                }
                __syncwarp();
            }

            if (ok) {
                // ---- streaming pass: transport (Step 3), classification, runs, flux sums
                const int n_tot = S.n_tot;
                const int ntouch = S.ntouch;
                StreamState st;
                st.pS = off;
                st.pL = off + slots;
                st.pR = off + 2 * static_cast<long long>(slots) - 1;
                st.acc = &S.acc[0][lane];
#pragma unroll
                for (int j = 0; j < 4; ++j) S.acc[j][lane] = 0;
                const StreamCtx ctx{&I, &E, ci, cell_base, g};
                if (S.staged) {
                    for (int base = 0; base < n_tot; base += 128) {
                        Rec v[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int k = base + 32 * u + lane;
                            if (k < n_tot) v[u] = ld_rec_rw(stage + k);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int k = base + 32 * u + lane;
                            if (base + 32 * u < n_tot) stream_group<Rec>(ctx, v[u], k < n_tot, k, out, fa, st);
                        }
                    }
                } else {
                    int tp = 0;   // first touched index not below the current group
                    for (int base = 0; base < n_in; base += 128) {
                        Rec v[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int k = base + 32 * u + lane;
                            if (k < n_in) v[u] = fetch_arrived<Rec>(k, nfb, fb, Rn, Rend, Sn, Sa, Ln, La, fa_, in, fs);
                        }
                        if (ntouch > 0) {
                            const int hi = min(base + 128, n_in);
                            for (int t = tp; t < ntouch && S.tidx[t] < hi; ++t) {
                                const int x = S.tidx[t];
                                const int u = (x - base) >> 5;
                                if (x >= base && (x & 31) == lane) {
#pragma unroll
                                    for (int uu = 0; uu < 4; ++uu)
                                        if (uu == u) v[uu] = S.trec[t];
                                }
                            }
                            while (tp < ntouch && S.tidx[tp] < hi) ++tp;
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int k = base + 32 * u + lane;
                            if (base + 32 * u < n_in) stream_group<Rec>(ctx, v[u], k < n_in, k, out, fa, st);
                        }
                    }
                    for (int base = n_in; base < n_tot; base += 32) {
                        const int k = base + lane;
                        Rec v;
                        if (k < n_tot) {
                            bool hit = false;
                            for (int t = tp; t < ntouch && S.tidx[t] < base + 32; ++t)
                                if (S.tidx[t] == k) { v = S.trec[t]; hit = true; }
                            if (!hit) v = sample_particle<Rec>(I, id, static_cast<uint32_t>(k - n_in), step, S.q);
                        }
                        stream_group<Rec>(ctx, v, k < n_tot, k, out, fa, st);
                        while (tp < ntouch && S.tidx[tp] < base + 32) ++tp;
                    }
                }
                __syncwarp();
                // moments of the L and R runs, read back with every lane busy
                const int nLr = static_cast<int>(st.pL - (off + slots));
                const int nRr = static_cast<int>(off + 2 * static_cast<long long>(slots) - 1 - st.pR);
                long long sLv[4] = {0, 0, 0, 0}, sRv[4] = {0, 0, 0, 0};
                run_sums<Rec>(out + off + slots, nLr, sLv, st.range_ok);
                run_sums<Rec>(out + st.pR + 1, nRr, sRv, st.range_ok);
                if (!__all_sync(0xffffffffu, st.range_ok) && lane == 0) set_err(E.err, kErrOverflow);
                long long rv[8] = {sLv[0], sLv[1], sLv[2], sLv[3], sRv[0], sRv[1], sRv[2], sRv[3]};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) rv[j] += __shfl_down_sync(0xffffffffu, rv[j], o);
                }
                int ngone = st.ngone;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ngone += __shfl_down_sync(0xffffffffu, ngone, o);
                long long gone = 0;
                if (lane < 4) {
                    for (int l = 0; l < 32; ++l) gone += S.acc[lane][l];
                }
                // lane j < 4 needs rv[j] and rv[4 + j] from lane 0
                long long lj = 0, rj = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long a0 = __shfl_sync(0xffffffffu, rv[j], 0);
                    const long long b0 = __shfl_sync(0xffffffffu, rv[4 + j], 0);
                    if (lane == j) { lj = a0; rj = b0; }
                }
                if (lane < 4) {
                    const double sc = (lane == 3) ? 0x1p-32 : 0x1p-40;
                    E.AL[4 * g + lane] = static_cast<double>(lj) * sc;
                    E.AR[4 * g + lane] = static_cast<double>(rj) * sc;
                    E.Aself[5 * g + 1 + lane] = static_cast<double>(gone - lj - rj) * sc;
                }
                if (lane == 0) {
                    E.Aself[5 * g] = -static_cast<double>(ngone + nLr + nRr);
                    S.nS = static_cast<int>(st.pS - off);
                    S.nL = static_cast<int>(st.pL - (off + slots));
                    S.nR = static_cast<int>(off + 2 * static_cast<long long>(slots) - 1 - st.pR);
                }
            } else if (lane == 0) {
                for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0.0; E.AR[4 * g + k] = 0.0; }
                for (int k = 0; k < 5; ++k) E.Aself[5 * g + k] = 0.0;
                S.skip = 1;
            }
        } else if (lane == 0) {
            for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0.0; E.AR[4 * g + k] = 0.0; }
            for (int k = 0; k < 5; ++k) E.Aself[5 * g + k] = 0.0;
        }
        __syncwarp();
        if (lane == 0) {
            const int done = !S.skip;
            if (done && !S.ghost) atomicAdd(&E.inst[S.b].updates, static_cast<unsigned long long>(S.n_tot));
            E.nL[wp][g] = done ? S.nL : 0;
            E.nS[wp][g] = done ? S.nS : 0;
            E.nR[wp][g] = done ? S.nR : 0;
            E.slotsb[wp][g] = done ? S.slots : 0;
            E.ncand[g] = done ? S.ncand : 0;
            E.nacc[g] = done ? S.nacc : 0;
            E.nabs[g] = done ? S.n_in - S.n_surv : 0;
            E.nnew[g] = done ? S.n_new : 0;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// Far movers: rank sort by (dest, src, q) -- keys are unique.
// ------------------------------------------------------------------------------------------
template <typename Rec>
__global__ void k_far_sort(EngineDev E)
{
    const FarItem<Rec> *a = static_cast<const FarItem<Rec> *>(E.far_app);
    FarItem<Rec> *s = static_cast<FarItem<Rec> *>(E.far_sorted);
    int n = *(volatile int32_t *)&E.far_count[0];
    if (n > E.far_cap) n = E.far_cap;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) E.far_count[1] = n;
    if (t >= n) return;
    const FarItem<Rec> me = a[t];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        const FarItem<Rec> &o = a[j];
        const bool less = (o.dest < me.dest) || (o.dest == me.dest && (o.src < me.src || (o.src == me.src && o.q < me.q)));
        rank += less ? 1 : 0;
    }
    s[rank] = me;
}

// ------------------------------------------------------------------------------------------
// Cell kernel: Eq. (r1) update, time average, primitive state, P, slot bound of the next step.
// ------------------------------------------------------------------------------------------
template <typename Rec>
__global__ void __launch_bounds__(kCellBlock) k_cells(EngineDev E, int q, int update)
{
    __shared__ int64_t s_w[kCellBlock / 32];
    const int g = blockIdx.x * kCellBlock + threadIdx.x;
    int64_t myslots = 0;
    if (threadIdx.x == 0 && blockIdx.x == 0 && update) E.far_count[0] = 0;
    if (g < E.G) {
        const int b = E.cell_inst[g];
        if (b >= 0) {
            const InstDev &I = E.inst[b];
            const int i = g - I.cell_base - 1;
            const uint32_t step_next = I.step + (update ? 1u : 0u);
            if (i < 0 || i >= I.C) {
                const int side = (i < 0) ? 0 : 1;
                const int bc = side ? I.bc_right : I.bc_left;
                if (bc == 0) {
                    double qg[5];
                    const bool ok = ghost_prim(I, side, qg, false, qg);
                    const double Pg = split_fraction(I, qg, ok);
                    myslots = ok ? resample_count(I, static_cast<uint32_t>(i + 1), step_next, Pg, qg[0]) : 0;
                }
                E.cnt[g] = 0;
            } else {
                // particles arriving in g and the sums of what they carry
                int farn = 0;
                double fsum[4] = {0, 0, 0, 0};
                const int nf = E.far_count[1];
                if (nf > 0) {
                    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
                    int lo = far_lower(fs, nf, g, INT32_MIN);
                    int hi = far_lower(fs, nf, g + 1, INT32_MIN);
                    farn = hi - lo;
                    for (int k = lo; k < hi; ++k) {
                        const double u = fs[k].rec.u, v = fs[k].rec.v, w = fs[k].rec.w;
                        fsum[0] += u; fsum[1] += v; fsum[2] += w; fsum[3] += 0.5 * (u * u + v * v + w * w);
                    }
                }
                const int arrivals = E.nR[q][g - 1] + E.nS[q][g] + E.nL[q][g + 1] + farn;
                double *psi = E.psi + 5 * g;
                if (update) {
                    const double *aR = E.AR + 4 * (g - 1), *aL = E.AL + 4 * (g + 1), *aS = E.Aself + 5 * g;
                    double dp[5];
                    dp[0] = static_cast<double>(E.nR[q][g - 1] + E.nL[q][g + 1] + farn) + aS[0];
                    for (int k = 0; k < 4; ++k) dp[k + 1] = aR[k] + aL[k] + fsum[k] + aS[k + 1];
                    const double *Fl = E.flux + 5 * (g - 1), *Fr = E.flux + 5 * g;
                    for (int k = 0; k < 5; ++k) {
                        const double fp = I.mp_over_dx * dp[k];
                        const double fw = I.dtdx * (Fr[k] - Fl[k]);
                        psi[k] = psi[k] + fp - fw;
                    }
                    if (static_cast<int64_t>(step_next) > static_cast<int64_t>(I.avg_start)) {
                        for (int k = 0; k < 5; ++k) E.avg[5 * g + k] += psi[k];
                    }
                }
                double qq[5];
                const bool ok = prim_from_cons(psi, I.R, qq);
                for (int k = 0; k < 5; ++k) E.prim[5 * g + k] = qq[k];
                E.valid[g] = ok ? 1 : 0;
                const double P = split_fraction(I, qq, ok);
                E.P[g] = P;
                int64_t extra = 0;
                if (ok) {
                    if (P == 0.0) {
                        extra = resample_count(I, static_cast<uint32_t>(i + 1), step_next, 0.0,
                                               psi[0] - static_cast<double>(arrivals) * I.mp_over_dx);
                    } else {
                        extra = static_cast<int64_t>(floor(((1.0 - P) * fmax(psi[0], 0.0)) * I.dx_over_mp)) + 2;
                    }
                }
                E.cnt[g] = arrivals;
                myslots = arrivals + extra;
            }
        }
        E.slots[g] = static_cast<int32_t>(myslots);
    }
    // block sum of the slot bounds
    int64_t x = myslots;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < kCellBlock / 32; ++w) s += s_w[w];
        E.blocksum[blockIdx.x] = 2 * s;
    }
}

// ------------------------------------------------------------------------------------------
// Offsets of the next step's output blocks and the wave flux of every interface.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kCellBlock) k_offsets_flux(EngineDev E, int wp, int advance)
{
    __shared__ int64_t s_w[kCellBlock / 32];
    __shared__ int64_t s_pre;
    const int g = blockIdx.x * kCellBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // sum of the slot bounds of all earlier blocks
    int64_t acc = 0;
    for (int j = threadIdx.x; j < blockIdx.x; j += kCellBlock) acc += E.blocksum[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) s_w[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < kCellBlock / 32; ++w) s += s_w[w];
        s_pre = s;
    }
    __syncthreads();
    // exclusive scan of the slots inside the block
    const int64_t v = (g < E.G) ? 2 * static_cast<int64_t>(E.slots[g]) : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    int64_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_w[w];
    if (g < E.G) {
        const int64_t o = s_pre + wpre + x - v;
        E.off[wp][g] = o;
        if (o + v > E.capacity) set_err(E.err, kErrOverflow);
    }
    if (g == 0) *E.ticket = 0;
    if (g >= E.G) return;
    const int b = E.cell_inst[g];
    if (b < 0) return;
    InstDev &I = E.inst[b];
    const int i = g - I.cell_base - 1;   // interface between local cells i and i+1
    if (i >= I.C) return;
    const int gl = (i < 0) ? -1 : g, gr = (i + 1 >= I.C) ? -1 : g + 1;
    double a[5], c[5];
    bool aok, cok;
    const bool periodic = (I.bc_left == 2);
    if (gl >= 0) { for (int k = 0; k < 5; ++k) a[k] = E.prim[5 * gl + k]; aok = E.valid[gl] != 0; }
    if (gr >= 0) { for (int k = 0; k < 5; ++k) c[k] = E.prim[5 * gr + k]; cok = E.valid[gr] != 0; }
    if (gl < 0) {
        if (periodic) {
            const int gg = I.cell_base + I.C;
            for (int k = 0; k < 5; ++k) a[k] = E.prim[5 * gg + k];
            aok = E.valid[gg] != 0;
        } else {
            aok = ghost_prim(I, 0, c, cok, a);
        }
    }
    if (gr < 0) {
        if (periodic) {
            const int gg = I.cell_base + 1;
            for (int k = 0; k < 5; ++k) c[k] = E.prim[5 * gg + k];
            cok = E.valid[gg] != 0;
        } else {
            cok = ghost_prim(I, 1, a, aok, c);
        }
    }
    wave_flux(I, a, aok, c, cok, E.flux + 5 * g);
    if (advance && i == -1) {
        const uint32_t nxt = I.step + 1u;
        if (static_cast<int64_t>(nxt) > static_cast<int64_t>(I.avg_start)) I.navg += 1;
        I.step = nxt;
    }
}

// ------------------------------------------------------------------------------------------
// Initial cells of one instance: all wave (Psi_p = 0), Psi_t from the two-state profile.
// ------------------------------------------------------------------------------------------
__global__ void k_init_cells(EngineDev E, int b, int g0, int n, double l0, double l1, double l2, double l3, double l4,
                             double r0, double r1, double r2, double r3, double r4, double x_min, double x_split)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int g = g0 + t;
    const InstDev &I = E.inst[b];
    E.cell_inst[g] = b;
    const int i = g - I.cell_base - 1;
    for (int p = 0; p < 2; ++p) { E.nL[p][g] = 0; E.nS[p][g] = 0; E.nR[p][g] = 0; E.off[p][g] = 0; E.slotsb[p][g] = 0; }
    for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0.0; E.AR[4 * g + k] = 0.0; }
    for (int k = 0; k < 5; ++k) { E.Aself[5 * g + k] = 0.0; E.avg[5 * g + k] = 0.0; E.flux[5 * g + k] = 0.0; E.psi[5 * g + k] = 0.0; E.prim[5 * g + k] = 0.0; }
    E.ncand[g] = 0; E.nacc[g] = 0; E.nabs[g] = 0; E.nnew[g] = 0; E.cnt[g] = 0; E.slots[g] = 0; E.valid[g] = 0; E.P[g] = 0.0; E.cmax[g] = 0.0; E.fmaj[g] = 1.0;
    if (i < 0 || i >= I.C) return;
    const double xc = x_min + (static_cast<double>(i) + 0.5) * I.dx;
    const bool left = xc < x_split;
    const double c[5] = {left ? l0 : r0, left ? l1 : r1, left ? l2 : r2, left ? l3 : r3, left ? l4 : r4};
    for (int k = 0; k < 5; ++k) E.psi[5 * g + k] = c[k];
    const double T = left ? I.left[4] : I.right[4];
    E.cmax[g] = 5.0 * sqrt(2.0 * I.R * T);
    E.fmaj[g] = majorant_factor(I, E.cmax[g]);
}

// ------------------------------------------------------------------------------------------
// Gather of the stable sorted list of instance b (inspection).
// ------------------------------------------------------------------------------------------
template <typename Rec>
__global__ void k_gather(EngineDev E, int rp, int g0, int ncell, const int64_t *start, int64_t total, int32_t *cell,
                         double *xl, double *u, double *v, double *w)
{
    const int t = blockIdx.x;
    if (t >= ncell) return;
    const int g = g0 + t;
    const Rec *in = static_cast<const Rec *>(E.buf[rp]);
    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
    const int nf = E.far_count[1];
    int lo = 0, mid = 0, hi = 0;
    if (nf > 0) {
        lo = far_lower(fs, nf, g, INT32_MIN);
        mid = far_lower(fs, nf, g, g + 2);
        hi = far_lower(fs, nf, g + 1, INT32_MIN);
    }
    const int64_t Rend = E.off[rp][g - 1] + 2 * static_cast<int64_t>(E.slotsb[rp][g - 1]);
    const int Rn = E.nR[rp][g - 1];
    const int64_t Sa = E.off[rp][g];
    const int Sn = E.nS[rp][g];
    const int64_t La = E.off[rp][g + 1] + E.slotsb[rp][g + 1];
    const int Ln = E.nL[rp][g + 1];
    const int nfb = mid - lo, nfa = hi - mid;
    const int n = nfb + Rn + Sn + Ln + nfa;
    const int64_t o = start[t];
    const int local = g - E.inst[E.cell_inst[g]].cell_base - 1;
    if (o + n > total) {
        if (threadIdx.x == 0) set_err(E.err, kErrOverflow);
        return;
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int r = k;
        Rec x;
        if (r < nfb) x = fs[lo + r].rec;
        else if ((r -= nfb) < Rn) x = in[Rend - 1 - r];
        else if ((r -= Rn) < Sn) x = in[Sa + r];
        else if ((r -= Sn) < Ln) x = in[La + r];
        else { r -= Ln; x = fs[mid + r].rec; }
        cell[o + k] = local;
        xl[o + k] = x.xl;
        u[o + k] = x.u;
        v[o + k] = x.v;
        w[o + k] = x.w;
    }
}

// ------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------
size_t particles_smem_bytes(int fp32, int threads)
{
    const size_t per = fp32 ? sizeof(WarpShared<RecF>) : sizeof(WarpShared<RecD>);
    return per * static_cast<size_t>(threads / 32);
}

template <typename K>
static int occupancy_of(K kern, int threads, size_t smem)
{
    int n = 0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int particles_occupancy(int fp32, int variant, int threads, size_t smem)
{
    if (variant && threads > 128) return 0;
    if (fp32) return variant ? occupancy_of(k_particles<RecF, 6>, threads, smem) : occupancy_of(k_particles<RecF, 1>, threads, smem);
    return variant ? occupancy_of(k_particles<RecD, 6>, threads, smem) : occupancy_of(k_particles<RecD, 1>, threads, smem);
}

cudaError_t launch_particles(const EngineDev &E, int fp32, int variant, int rp, int grid, int threads, size_t smem,
                             cudaStream_t s)
{
    if (fp32) {
        if (variant) k_particles<RecF, 6><<<grid, threads, smem, s>>>(E, rp);
        else k_particles<RecF, 1><<<grid, threads, smem, s>>>(E, rp);
    } else {
        if (variant) k_particles<RecD, 6><<<grid, threads, smem, s>>>(E, rp);
        else k_particles<RecD, 1><<<grid, threads, smem, s>>>(E, rp);
    }
    return cudaGetLastError();
}

cudaError_t launch_far_sort(const EngineDev &E, int fp32, cudaStream_t s)
{
    const int grid = (E.far_cap + 255) / 256;
    if (fp32) k_far_sort<RecF><<<grid, 256, 0, s>>>(E);
    else k_far_sort<RecD><<<grid, 256, 0, s>>>(E);
    return cudaGetLastError();
}

cudaError_t launch_cells(const EngineDev &E, int fp32, int q, int update, cudaStream_t s)
{
    const int grid = (E.G + kCellBlock - 1) / kCellBlock;
    if (fp32) k_cells<RecF><<<grid, kCellBlock, 0, s>>>(E, q, update);
    else k_cells<RecD><<<grid, kCellBlock, 0, s>>>(E, q, update);
    return cudaGetLastError();
}

cudaError_t launch_offsets_flux(const EngineDev &E, int wp, int advance, cudaStream_t s)
{
    const int grid = (E.G + kCellBlock - 1) / kCellBlock;
    k_offsets_flux<<<grid, kCellBlock, 0, s>>>(E, wp, advance);
    return cudaGetLastError();
}

cudaError_t launch_init_cells(const EngineDev &E, int b, int g0, int n, const double *lc, const double *rc, double x_min,
                              double x_split, cudaStream_t s)
{
    const int grid = (n + 255) / 256;
    k_init_cells<<<grid, 256, 0, s>>>(E, b, g0, n, lc[0], lc[1], lc[2], lc[3], lc[4], rc[0], rc[1], rc[2], rc[3], rc[4],
                                      x_min, x_split);
    return cudaGetLastError();
}

cudaError_t launch_gather(const EngineDev &E, int fp32, int rp, int b, int g0, int ncell, const int64_t *d_start,
                          int64_t total, int32_t *cell, double *xl, double *u, double *v, double *w, cudaStream_t s)
{
    (void)b;
    if (ncell <= 0) return cudaSuccess;
    if (fp32) k_gather<RecF><<<ncell, 128, 0, s>>>(E, rp, g0, ncell, d_start, total, cell, xl, u, v, w);
    else k_gather<RecD><<<ncell, 128, 0, s>>>(E, rp, g0, ncell, d_start, total, cell, xl, u, v, w);
    return cudaGetLastError();
}

}  // namespace duwp

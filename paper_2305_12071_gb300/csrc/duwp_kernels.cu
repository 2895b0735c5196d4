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
__device__ inline Rec sample_particle(const InstDev &I, uint32_t id, uint32_t j, uint32_t step, const double *q)
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
template <typename Rec>
__device__ void collide_warp(const InstDev &I, uint32_t id, uint32_t step, Rec *list, int N, double rho_t,
                             double &cmax, int &ncand, int &nacc, int *s_ab)
{
    using T = decltype(list[0].xl);
    const int lane = threadIdx.x & 31;
    ncand = 0;
    nacc = 0;
    if (N < 2) return;
    const double rr = (I.ntc_rate == 1) ? rho_t / I.rho_ref : ((static_cast<double>(N) * I.mp) / I.dx) / I.rho_ref;
    const double f = (I.upsilon == 0.0) ? 1.0 : pow(cmax / I.c_ref, -2.0 * I.upsilon);
    const double nsel = I.ntc_A * rr * (static_cast<double>(N) - 1.0) * f * cmax;
    uint32_t w[4];
    draw(I, id, 1u, step, kRound, w);
    int64_t nc = static_cast<int64_t>(floor(nsel + u53(w[0], w[1])));
    if (!(nsel < 1e8)) { ncand = -1; return; }
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
        double cr = 0.0;
        if (lane < m1) {
            A = list[a];
            B = list[b];
            const double d0 = static_cast<double>(A.u) - static_cast<double>(B.u);
            const double d1 = static_cast<double>(A.v) - static_cast<double>(B.v);
            const double d2 = static_cast<double>(A.w) - static_cast<double>(B.w);
            cr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        }
        const unsigned rmask = __ballot_sync(0xffffffffu, lane < m1 && cr > cm);
        const int fr = rmask ? __ffs(rmask) - 1 : 32;
        const int m = min(m1, fr + 1);
        const double cr_r = __shfl_sync(0xffffffffu, cr, fr < 32 ? fr : 0);
        bool accd = false;
        if (lane < m) {
            const double cml = (lane == fr) ? cr : cm;
            const double x = cr / cml;
            if (I.upsilon == 0.0) {
                accd = ua < x;
            } else if (expo == 0.0) {
                accd = ua < 1.0;
            } else {
                const float pf = exp2f(expo_f * log2f(static_cast<float>(x)));
                const double p = static_cast<double>(pf);
                const double margin = 2e-5 * p;
                if (ua < p - margin) accd = true;
                else if (ua > p + margin) accd = false;
                else accd = ua < pow(x, expo);
            }
            if (accd) {
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
                list[a] = A;
                list[b] = B;
            }
        }
        acc += __popc(__ballot_sync(0xffffffffu, accd));
        if (fr < m) cm = cr_r;
        __syncwarp();
        k0 += m;
    }
    cmax = cm;
    ncand = static_cast<int>(nc);
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
// Particle kernel
// ------------------------------------------------------------------------------------------
struct CellHdr {
    int b, i, ghost, skip;
    int n_in, slots, n_surv, n_new, n_tot;
    int nfb, nfa, fb, fa;
    long long Ra, Sa, La, off_out;
    int Rn, Sn, Ln;
    double P, rho_t, cmax;
    double q[5];
    int valid;
    int ncand, nacc;
    int nL, nS, nR;
};

constexpr int kMaxWarps = 16;

struct PartShared {
    CellHdr H;
    int g;
    int wcnt[kMaxWarps][3];
    long long red[kMaxWarps][13];
    uint64_t scan[32];
    uint64_t run;
    int ab[64];
};

// Stages of one cell after the header: list = the cell's staging area (shared memory or a
// global slice), cls = one byte per particle.
template <typename Rec>
__device__ __forceinline__ void process_cell(const EngineDev &E, int rp, int g, PartShared &S, Rec *__restrict__ list,
                                             uint8_t *__restrict__ cls)
{
    using T = decltype(Rec().xl);
    CellHdr &H = S.H;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int wp = 1 - rp;
    const Rec *in = static_cast<const Rec *>(E.buf[rp]);
    Rec *out = static_cast<Rec *>(E.buf[wp]);
    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
    FarItem<Rec> *fa = static_cast<FarItem<Rec> *>(E.far_app);
    const InstDev &I = E.inst[H.b];
    const uint32_t step = I.step;
    const uint32_t id = static_cast<uint32_t>(H.i + 1);

    // ---------------- gather the arrived list (sorted order) into the staging area
    const int n_in = H.n_in;
    for (int k = tid; k < n_in; k += nt) {
        int r = k;
        Rec v;
        if (r < H.nfb) { v = fs[H.fb + r].rec; }
        else if ((r -= H.nfb) < H.Rn) { v = ld_rec(in + H.Ra + r); }
        else if ((r -= H.Rn) < H.Sn) { v = ld_rec(in + H.Sa + r); }
        else if ((r -= H.Sn) < H.Ln) { v = ld_rec(in + H.La + r); }
        else { r -= H.Ln; v = fs[H.fa + r].rec; }
        list[k] = v;
    }
    __syncthreads();

    // ---------------- absorption into the wave with probability P (Eq. p), stable compaction
    int n_surv = n_in;
    if (!H.ghost && H.P > 0.0) {
        const double P = H.P;
        if (tid == 0) S.run = 0;
        __syncthreads();
        for (int base = 0; base < n_in; base += nt) {
            const int k = base + tid;
            Rec v;
            int keep = 0;
            if (k < n_in) {
                v = list[k];
                uint32_t w[4];
                draw(I, id, static_cast<uint32_t>(k), step, kAbsorb, w);
                keep = !(u53(w[0], w[1]) < P);
            }
            uint64_t tot;
            const uint64_t pos = block_scan_u64(static_cast<uint64_t>(keep), S.scan, &tot);
            const uint64_t run = S.run;
            __syncthreads();
            if (keep) list[run + pos] = v;
            __syncthreads();
            if (tid == 0) S.run = run + tot;
            __syncthreads();
        }
        n_surv = static_cast<int>(S.run);
    }

    // ---------------- re-sampling of (1-P) of the wave (Step 2)
    if (tid == 0) {
        H.n_surv = n_surv;
        if (!H.ghost) {
            const double rho_w = H.rho_t - static_cast<double>(n_surv) * I.mp_over_dx;
            H.n_new = H.valid ? static_cast<int>(resample_count(I, id, step, H.P, rho_w)) : 0;
        }
        H.n_tot = n_surv + H.n_new;
        if (H.n_tot > H.slots || H.off_out + H.n_tot > E.capacity) {
            set_err(E.err, kErrOverflow);
            H.skip = 1;
        }
    }
    __syncthreads();
    if (H.skip) return;
    const int n_tot = H.n_tot;
    for (int j = tid; j < H.n_new; j += nt) list[n_surv + j] = sample_particle<Rec>(I, id, static_cast<uint32_t>(j), step, H.q);
    __syncthreads();

    // ---------------- collisions (Appendix A), one warp
    if (!H.ghost && warp == 0) {
        double cmax = H.cmax;
        int nc = 0, na = 0;
        collide_warp<Rec>(I, id, step, list, n_tot, H.rho_t, cmax, nc, na, S.ab);
        if (lane == 0) {
            if (nc < 0) { set_err(E.err, kErrOverflow); nc = 0; }
            H.ncand = nc;
            H.nacc = na;
            E.cmax[g] = cmax;
        }
    }
    __syncthreads();

    // ---------------- transport, classification and flux sums (pass A, one chunk per warp)
    const int chunk = (((n_tot + nw - 1) / nw) + 31) & ~31;
    const int c0 = min(warp * chunk, n_tot), c1 = min(c0 + chunk, n_tot);
    long long sL[4] = {0, 0, 0, 0}, sR[4] = {0, 0, 0, 0}, sS[4] = {0, 0, 0, 0};
    int nlv = 0, cntL = 0, cntS = 0, cntR = 0;
    const int cell_base = I.cell_base;
    for (int base = c0; base < c1; base += 32) {
        const int k = base + lane;
        int c = 5;
        if (k < c1) {
            Rec v = list[k];
            const T u0 = v.u;
            T xl = v.xl, uu = v.u;
            bool refl = false;
            const int64_t d = transport(I, H.i, xl, uu, refl);
            v.xl = xl;
            v.u = uu;
            if (d < 0) c = 4;
            else if (d == H.i - 1) c = 0;
            else if (d == H.i) c = 1;
            else if (d == H.i + 1) c = 2;
            else c = 3;
            if (!(fx_in_range(u0) && fx_in_range(v.v) && fx_in_range(v.w))) set_err(E.err, kErrOverflow);
            if (c == 1) {
                if (refl) sS[0] += fx_vel(uu) - fx_vel(u0);
            } else {
                const long long qv = fx_vel(v.v), qw = fx_vel(v.w), qe = fx_energy(u0, v.v, v.w);
                ++nlv;
                sS[0] -= fx_vel(u0); sS[1] -= qv; sS[2] -= qw; sS[3] -= qe;
                if (c == 0) { sL[0] += fx_vel(uu); sL[1] += qv; sL[2] += qw; sL[3] += qe; }
                else if (c == 2) { sR[0] += fx_vel(uu); sR[1] += qv; sR[2] += qw; sR[3] += qe; }
                else if (c == 3) {
                    const int slot = atomicAdd(&E.far_count[0], 1);
                    if (slot < E.far_cap) {
                        FarItem<Rec> it;
                        it.dest = cell_base + 1 + static_cast<int>(d);
                        it.src = g;
                        it.q = k;
                        it.pad = 0;
                        it.rec = v;
                        fa[slot] = it;
                    } else {
                        set_err(E.err, kErrOverflow);
                    }
                }
            }
            list[k] = v;
            cls[k] = static_cast<uint8_t>(c);
        }
        cntL += __popc(__ballot_sync(0xffffffffu, c == 0));
        cntS += __popc(__ballot_sync(0xffffffffu, c == 1));
        cntR += __popc(__ballot_sync(0xffffffffu, c == 2));
    }
    // per-warp class counts and moment sums
    {
        long long vals[13] = {sL[0], sL[1], sL[2], sL[3], sR[0], sR[1], sR[2], sR[3],
                              sS[0], sS[1], sS[2], sS[3], static_cast<long long>(nlv)};
#pragma unroll
        for (int j = 0; j < 13; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vals[j] += __shfl_down_sync(0xffffffffu, vals[j], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < 13; ++j) S.red[warp][j] = vals[j];
            S.wcnt[warp][0] = cntL;
            S.wcnt[warp][1] = cntS;
            S.wcnt[warp][2] = cntR;
        }
    }
    __syncthreads();
    if (tid < 13) {
        long long s = 0;
        for (int w2 = 0; w2 < nw; ++w2) s += S.red[w2][tid];
        if (tid < 4) E.AL[4 * g + tid] = static_cast<double>(s) * (tid < 3 ? 0x1p-40 : 0x1p-32);
        else if (tid < 8) E.AR[4 * g + tid - 4] = static_cast<double>(s) * (tid < 7 ? 0x1p-40 : 0x1p-32);
        else if (tid < 12) E.Aself[5 * g + tid - 7] = static_cast<double>(s) * (tid < 11 ? 0x1p-40 : 0x1p-32);
        else E.Aself[5 * g] = -static_cast<double>(s);
    }
    // warp bases of the three runs
    int wbL = 0, wbS = 0, wbR = 0, tL = 0, tS = 0, tR = 0;
    for (int w2 = 0; w2 < nw; ++w2) {
        const int a0 = S.wcnt[w2][0], a1 = S.wcnt[w2][1], a2 = S.wcnt[w2][2];
        if (w2 < warp) { wbL += a0; wbS += a1; wbR += a2; }
        tL += a0; tS += a1; tR += a2;
    }
    // ---------------- stable partition into the output block [L | S | R] (pass B, no barriers)
    long long pL = H.off_out + wbL, pS = H.off_out + tL + wbS, pR = H.off_out + tL + tS + wbR;
    const unsigned lt = (1u << lane) - 1u;
    for (int base = c0; base < c1; base += 32) {
        const int k = base + lane;
        const int c = (k < c1) ? cls[k] : 5;
        const unsigned mL = __ballot_sync(0xffffffffu, c == 0);
        const unsigned mS = __ballot_sync(0xffffffffu, c == 1);
        const unsigned mR = __ballot_sync(0xffffffffu, c == 2);
        if (c <= 2) {
            const unsigned mm = (c == 0) ? mL : (c == 1) ? mS : mR;
            const long long pb = (c == 0) ? pL : (c == 1) ? pS : pR;
            st_rec(out + pb + __popc(mm & lt), list[k]);
        }
        pL += __popc(mL);
        pS += __popc(mS);
        pR += __popc(mR);
    }
    if (tid == 0) {
        H.nL = tL;
        H.nS = tS;
        H.nR = tR;
    }
}

// kMinBlocks = 1: registers unconstrained (up to 512 threads per block); kMinBlocks = 6: at most
// 128 threads and about 80 registers per thread, so that six blocks fit on one SM.
template <typename Rec, int kMinBlocks>
__global__ void __launch_bounds__(kMinBlocks == 1 ? 512 : 128, kMinBlocks) k_particles(EngineDev E, int rp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Rec *sm = reinterpret_cast<Rec *>(smraw);
    uint8_t *smcls = smraw + static_cast<size_t>(E.cell_cap) * sizeof(Rec);
    __shared__ PartShared S;
    CellHdr &H = S.H;
    const int wp = 1 - rp;
    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
    const int tid = threadIdx.x;
    Rec *gstage = static_cast<Rec *>(E.stage) + static_cast<size_t>(blockIdx.x) * E.stage_cap;
    uint8_t *gcls = E.stage_cls + static_cast<size_t>(blockIdx.x) * E.stage_cap;

    for (;;) {
        if (tid == 0) S.g = atomicAdd(E.ticket, 1);
        __syncthreads();
        const int g = S.g;
        if (g >= E.G) break;

        // ---------------- header (one thread)
        if (tid == 0) {
            H.skip = 0;
            H.b = E.cell_inst[g];
            H.ncand = H.nacc = 0;
            H.nL = H.nS = H.nR = 0;
            H.n_in = H.n_surv = H.n_new = H.n_tot = 0;
            H.nfb = H.nfa = 0;
            H.Rn = H.Sn = H.Ln = 0;
            if (H.b < 0) {
                H.skip = 1;
            } else {
                const InstDev &I = E.inst[H.b];
                H.i = g - I.cell_base - 1;
                H.ghost = (H.i < 0) ? 1 : (H.i >= I.C ? 2 : 0);
                H.slots = E.slots[g];
                H.off_out = E.off[wp][g];
                if (H.ghost) {
                    const int side = H.ghost - 1;
                    const int bc = side ? I.bc_right : I.bc_left;
                    if (bc != 0) {
                        H.skip = 1;
                    } else {
                        double q[5];
                        const bool ok = ghost_prim(I, side, q, false, q);
                        for (int k = 0; k < 5; ++k) H.q[k] = q[k];
                        H.valid = ok;
                        H.P = split_fraction(I, q, ok);
                        H.rho_t = 0.0;
                        H.cmax = 0.0;
                        H.n_new = ok ? static_cast<int>(resample_count(I, static_cast<uint32_t>(H.i + 1), I.step, H.P, q[0])) : 0;
                    }
                } else {
                    for (int k = 0; k < 5; ++k) H.q[k] = E.prim[5 * g + k];
                    H.valid = E.valid[g];
                    H.P = E.P[g];
                    H.rho_t = E.psi[5 * g];
                    H.cmax = E.cmax[g];
                    H.Ra = E.off[rp][g - 1] + E.nL[rp][g - 1] + E.nS[rp][g - 1];
                    H.Rn = E.nR[rp][g - 1];
                    H.Sa = E.off[rp][g] + E.nL[rp][g];
                    H.Sn = E.nS[rp][g];
                    H.La = E.off[rp][g + 1];
                    H.Ln = E.nL[rp][g + 1];
                    const int nf = E.far_count[1];
                    int lo = 0, mid = 0, hi = 0;
                    if (nf > 0) {
                        lo = far_lower(fs, nf, g, INT32_MIN);
                        mid = far_lower(fs, nf, g, g + 2);
                        hi = far_lower(fs, nf, g + 1, INT32_MIN);
                    }
                    H.fb = lo;
                    H.nfb = mid - lo;
                    H.fa = mid;
                    H.nfa = hi - mid;
                    H.n_in = H.nfb + H.Rn + H.Sn + H.Ln + H.nfa;
                    if (H.n_in != E.cnt[g] || H.n_in > H.slots) {
                        set_err(E.err, kErrOverflow);
                        H.skip = 1;
                    }
                }
                if (!H.skip && H.slots > E.cell_cap && H.slots > E.stage_cap) {
                    set_err(E.err, kErrOverflow);
                    H.skip = 1;
                }
            }
        }
        __syncthreads();
        if (!H.skip) {
            if (H.slots <= E.cell_cap) process_cell<Rec>(E, rp, g, S, sm, smcls);
            else process_cell<Rec>(E, rp, g, S, gstage, gcls);
        }
        __syncthreads();
        if (tid == 0) {
            const int done = !H.skip;
            if (done && !H.ghost) atomicAdd(&E.inst[H.b].updates, static_cast<unsigned long long>(H.n_tot));
            E.nL[wp][g] = done ? H.nL : 0;
            E.nS[wp][g] = done ? H.nS : 0;
            E.nR[wp][g] = done ? H.nR : 0;
            E.ncand[g] = done ? H.ncand : 0;
            E.nacc[g] = done ? H.nacc : 0;
            E.nabs[g] = done ? H.n_in - H.n_surv : 0;
            E.nnew[g] = done ? H.n_new : 0;
            if (!done) {
                for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0.0; E.AR[4 * g + k] = 0.0; }
                for (int k = 0; k < 5; ++k) E.Aself[5 * g + k] = 0.0;
            }
        }
        __syncthreads();
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
        E.blocksum[blockIdx.x] = s;
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
    const int64_t v = (g < E.G) ? E.slots[g] : 0;
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
    for (int p = 0; p < 2; ++p) { E.nL[p][g] = 0; E.nS[p][g] = 0; E.nR[p][g] = 0; E.off[p][g] = 0; }
    for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0.0; E.AR[4 * g + k] = 0.0; }
    for (int k = 0; k < 5; ++k) { E.Aself[5 * g + k] = 0.0; E.avg[5 * g + k] = 0.0; E.flux[5 * g + k] = 0.0; E.psi[5 * g + k] = 0.0; E.prim[5 * g + k] = 0.0; }
    E.ncand[g] = 0; E.nacc[g] = 0; E.nabs[g] = 0; E.nnew[g] = 0; E.cnt[g] = 0; E.slots[g] = 0; E.valid[g] = 0; E.P[g] = 0.0; E.cmax[g] = 0.0;
    if (i < 0 || i >= I.C) return;
    const double xc = x_min + (static_cast<double>(i) + 0.5) * I.dx;
    const bool left = xc < x_split;
    const double c[5] = {left ? l0 : r0, left ? l1 : r1, left ? l2 : r2, left ? l3 : r3, left ? l4 : r4};
    for (int k = 0; k < 5; ++k) E.psi[5 * g + k] = c[k];
    const double T = left ? I.left[4] : I.right[4];
    E.cmax[g] = 5.0 * sqrt(2.0 * I.R * T);
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
    const int64_t Ra = E.off[rp][g - 1] + E.nL[rp][g - 1] + E.nS[rp][g - 1];
    const int Rn = E.nR[rp][g - 1];
    const int64_t Sa = E.off[rp][g] + E.nL[rp][g];
    const int Sn = E.nS[rp][g];
    const int64_t La = E.off[rp][g + 1];
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
        else if ((r -= nfb) < Rn) x = in[Ra + r];
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
size_t particles_smem_bytes(int fp32, int cell_cap)
{
    const size_t rec = fp32 ? sizeof(RecF) : sizeof(RecD);
    size_t b = static_cast<size_t>(cell_cap) * rec + static_cast<size_t>(cell_cap);
    return (b + 15) & ~static_cast<size_t>(15);
}

static size_t static_smem_particles()
{
    return sizeof(PartShared) + 64;
}

int max_cell_capacity(int fp32)
{
    const size_t limit = 227 * 1024 - static_smem_particles();
    const size_t per = (fp32 ? sizeof(RecF) : sizeof(RecD)) + 1;
    return static_cast<int>((limit - 16) / per);
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

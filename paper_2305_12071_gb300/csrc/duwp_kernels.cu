// duwp_kernels.cu -- the per-step kernels of the DUWP method (arXiv 2305.12071, Sec. 3.4) on sm_103a.
//
//   k_collide     (persistent, one warp per listed cell): NTC/VHS collisions (Appendix A) of the
//                 cells that have candidates, and absorption with probability P (Eq. p) plus
//                 re-sampling of (1-P) of the wave (Eq. maxsample) in the cells where P > 0.
//   k_stream      (one warp per cell): read the cell's stable list (far movers, R(g-1), S(g),
//                 L(g+1), or the staged list), sample the re-sampled particles of cells without
//                 collisions, free transport with boundaries (Step 3), write the L/S/R runs of the
//                 cell's output block, exact sums of the moments that left or entered (Eq. fp).
//   k_far_sort    stable order of the rare particles that moved two or more cells.
//   k_cells       (per cell): conservative update Eq. (r1), time average, primitive state, P, the
//                 slot bound and the plan (counts, class) of the next step.
//   k_offsets     (per cell): output block offsets of the next step (scan of the slot bounds), the
//                 work lists of the collision kernels.
//   k_flux        (per interface): the wave flux from the cell kernel's states, at the start of the
//                 step that applies it, beside that step's particle kernels.
#include <algorithm>
#include <type_traits>
#include <cstdio>

#include "duwp_dsmath.cuh"
#include "duwp_launch.h"

namespace duwp {

// cos and sin of 2 pi k / kTurnTable as double-single pairs (scattering and sampling of
// single-precision records), and the log table of the sampling (1/F and log F at F = 1 + (j - kLogCenter)/1024)
__device__ float4 g_turn[kTurnTable];
__device__ float4 g_logt[kLogTable];

__device__ __forceinline__ float2 ds_split(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - static_cast<double>(h)));
}

__global__ void k_init_turn()
{
    const int k = threadIdx.x;
    if (k < kTurnTable) {
        double s, c;
        sincospi(static_cast<double>(k) / (0.5 * kTurnTable), &s, &c);
        const float2 cc = ds_split(c), ss = ds_split(s);
        g_turn[k] = make_float4(cc.x, cc.y, ss.x, ss.y);
    }
    if (k < kLogTable) {
        const double F = static_cast<double>(1024 + k - kLogCenter) * 0x1p-10;
        const float2 inv = ds_split(1.0 / F), lg = ds_split(log(F));
        g_logt[k] = make_float4(inv.x, inv.y, lg.x, lg.y);
    }
}

// Programmatic dependent launch: the step's kernels are launched with programmatic stream
// serialization, so that a kernel's blocks are scheduled while its predecessor's last blocks finish;
// every step kernel first waits here until the predecessor grid has completed and its memory is
// visible (a no-op where the launch had no programmatic dependency).
__device__ __forceinline__ void wait_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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
        if ((dest < 0 && I.bc_left == kBcPhantom) || (dest >= C && I.bc_right == kBcPhantom))
            return dest;     // into another part of the domain (phantom side): kept, exported
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
            return kGone;
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
            return kGone;
        }
        return dest;
    }
    return kGone;   // more than 64 wall reflections within one step: removed
}

__device__ __forceinline__ int64_t transport(const InstDev &I, int64_t cell, double &xl, double &u, bool &refl)
{
    const double s = __fma_rn(u, I.dtdx, xl);
    if (!(fabs(s) < 1e15)) return kGone;
    const double fk = floor(s);
    double x = __dsub_rn(s, fk);
    int64_t k = static_cast<int64_t>(fk);
    if (x >= 1.0) { x = 0.0; k += 1; }
    xl = x;
    return apply_walls<double>(I, cell + k, xl, u, refl);
}

// ------------------------------------------------------------------------------------------
// Maxwellian sample at the primitive state q (Eq. maxsample) by Box-Muller pairs: radius
// sqrt(2RT) sqrt(-ln r2), r2 in (0,1], angle 2 pi r1 -> x (cosine) and y (sine); z from its own pair
// (r3, r4) and its cosine; position uniform in the cell.  Particle j of a cell uses counters
// (id, 4j..4j+2, step, SAMPLE): uniforms 0 -> position, 1 -> r1, 2 -> r2, 3 -> r3, 4 -> r4.
// ------------------------------------------------------------------------------------------
// Per-cell part of the sample: the state and sqrt(2RT), also as double-single values.
struct MaxwellCell {
    double q[5];
    double sq;
    ds U[3];
    ds s;
    const double *qp;       // the cell's primitive state (rho, U, V, W, T) in device memory
};

// Chapman-Enskog factor of a cell's samples under the NS-corrected option (below).
struct CeCell {
    double A, sxx, syy, sxy, sxz, qx, prt, RT;
};

__device__ inline MaxwellCell maxwell_cell(const InstDev &I, const double *q)
{
    MaxwellCell m;
    m.qp = q;
    for (int k = 0; k < 5; ++k) m.q[k] = q[k];
    m.sq = sqrt(2.0 * I.R * q[4]);
    for (int d = 0; d < 3; ++d) {
        const float h = __double2float_rn(q[1 + d]);
        m.U[d] = {h, __double2float_rn(q[1 + d] - static_cast<double>(h))};
    }
    const float h = __double2float_rn(m.sq);
    m.s = {h, __double2float_rn(m.sq - static_cast<double>(h))};
    return m;
}

// The sampling state of a cell for single-precision records drawn without the NS correction: only
// the double-single U and s, formed by integer and single-precision operations (the double-precision
// units are few on this GPU and a chunk of draws is short); q and sq are not set, and a draw that
// takes the double-precision path reads the state from qp.  Double-precision records (and values
// outside the integer conversion's range) take the full state.
template <typename Rec>
__device__ inline MaxwellCell maxwell_cell_for(const InstDev &I, const double *q)
{
    if constexpr (sizeof(Rec) == sizeof(RecF)) {
        MaxwellCell m;
        m.qp = q;
        if (ds_maxwell_params(I.R, q, m.U, m.s)) return m;
    }
    return maxwell_cell(I, q);
}

// Velocities in double precision from the 8 draw words after the position's (w), by the Box-Muller
// transform: the angle 2 pi r1 and the radius sqrt(2RT) sqrt(-ln r2) give the x component (cosine)
// and the y component (sine); z takes its own angle r3 and radius r4 (cosine).
__device__ __forceinline__ void maxwell_xi(const MaxwellCell &mc, const uint32_t *w, double out[3])
{
    const double r1 = u53(w[0], w[1]);
    const double r2 = 1.0 - u53(w[2], w[3]);
    const double r3 = u53(w[4], w[5]);
    const double r4 = 1.0 - u53(w[6], w[7]);
    const double rad = sqrt(-log(r2));
    out[0] = mc.q[1] + (mc.sq * cos(kTwoPi * r1)) * rad;
    out[1] = mc.q[2] + (mc.sq * sin(kTwoPi * r1)) * rad;
    out[2] = mc.q[3] + (mc.sq * cos(kTwoPi * r3)) * sqrt(-log(r4));
}

template <typename T>
__device__ __noinline__ void maxwell_fp64(const MaxwellCell &mc, const uint32_t *w, T out[3])
{
    double xi[3];
    maxwell_xi(mc, w, xi);
#pragma unroll
    for (int d = 0; d < 3; ++d) out[d] = store_val(xi[d], T());
}

// The same double-precision evaluation for a single-precision record from the cell's state in memory
// (words w[2..9] of the draw by value, so that the caller keeps them in registers); returns the
// record's velocities in y, z, w.
__device__ __noinline__ float4 maxwell_fp64_from(double R, const double *q, uint4 wa, uint4 wb)
{
    const double sq = sqrt(2.0 * R * q[4]);
    const double r1 = u53(wa.x, wa.y);
    const double r2 = 1.0 - u53(wa.z, wa.w);
    const double r3 = u53(wb.x, wb.y);
    const double r4 = 1.0 - u53(wb.z, wb.w);
    const double rad = sqrt(-log(r2));
    return make_float4(0.0f, __double2float_rn(q[1] + (sq * cos(kTwoPi * r1)) * rad),
                       __double2float_rn(q[2] + (sq * sin(kTwoPi * r1)) * rad),
                       __double2float_rn(q[3] + (sq * cos(kTwoPi * r3)) * sqrt(-log(r4))));
}

// NS-corrected sampling (resample_mode CE; the first-order Chapman-Enskog form of the equilibrium,
// Eq. ce2): the density f_M (1 + sigma_ij c_i c_j / (2 p R T) + (q . c / (p R T)) (c^2 / (5 R T) - 1)),
// c = xi - U, with the 1D NS stress and heat flux of the wave at the viscosity eps mu of its flux
// (Eq. vp1, Sec. 3.3):
//   sigma_xx = -(4/3) mu_e dU/dx, sigma_yy = sigma_zz = (2/3) mu_e dU/dx, sigma_xy = -mu_e dV/dx,
//   sigma_xz = -mu_e dW/dx, q_x = -kappa_e dT/dx, kappa_e = (5/2) R mu_e / Pr,
// the gradients by central differences of the neighbouring states (the periodic partner or the
// reservoir/mirror state beyond an end; an unusable neighbour counts as the cell's own state).
// Drawn by acceptance-rejection against A = 1 + 30 B, B the largest of |sigma_ij| / p and
// 2 |q_x| / (p sqrt(2RT)) (Garcia and Alder, J. Comput. Phys. 140, 1998); for B > 1/4 the expansion
// is out of range and the plain Maxwellian is drawn.  Every expression keeps the order of
// operations of the double-precision checker, so decisions agree to the last bit of the inputs.
constexpr int kCeAttempts = 64;

// Returns false where the plain Maxwellian is drawn.
__device__ __noinline__ bool ce_coefs(const InstDev &I, const double *prim, const int32_t *valid, int g, int i,
                                      CeCell &m)
{
    if (!valid[g]) return false;
    const double *W0 = prim + 5 * g;
    double wm[5], wp[5];
    bool okm, okp;
    const bool periodic = (I.bc_left == 2);
    if (i > 0 || I.bc_left == kBcPhantom) { for (int k = 0; k < 5; ++k) wm[k] = W0[k - 5]; okm = valid[g - 1] != 0; }
    else if (periodic) { for (int k = 0; k < 5; ++k) wm[k] = prim[5 * (g + I.C - 1) + k]; okm = valid[g + I.C - 1] != 0; }
    else okm = ghost_prim(I, 0, W0, true, wm);
    if (i < I.C - 1 || I.bc_right == kBcPhantom) { for (int k = 0; k < 5; ++k) wp[k] = W0[k + 5]; okp = valid[g + 1] != 0; }
    else if (periodic) { for (int k = 0; k < 5; ++k) wp[k] = prim[5 * (g - I.C + 1) + k]; okp = valid[g - I.C + 1] != 0; }
    else okp = ghost_prim(I, 1, W0, true, wp);
    const double *a = okm ? wm : W0, *b = okp ? wp : W0;
    const double inv = 1.0 / (2.0 * I.dx);
    const double dU = (b[1] - a[1]) * inv, dV = (b[2] - a[2]) * inv, dW = (b[3] - a[3]) * inv;
    const double dT = (b[4] - a[4]) * inv;
    const double RT = I.R * W0[4];
    const double p0 = W0[0] * RT;
    const double mu = viscosity(I, W0[4]);
    const double mue = eps_factor(I.eps_mode, I.dt / (mu / p0)) * mu;
    const double kap = 2.5 * I.R * mue / I.Pr;
    m.sxx = -(4.0 / 3.0) * mue * dU;
    m.syy = (2.0 / 3.0) * mue * dU;
    m.sxy = -mue * dV;
    m.sxz = -mue * dW;
    m.qx = -kap * dT;
    double B = fmax(fmax(fabs(m.sxx), fabs(m.syy)), fmax(fabs(m.sxy), fabs(m.sxz))) / p0;
    B = fmax(B, 2.0 * fabs(m.qx) / (p0 * sqrt(2.0 * RT)));
    if (!(B <= 0.25)) return false;
    m.RT = RT;
    m.prt = p0 * RT;
    m.A = 1.0 + 30.0 * B;
    return true;
}

__device__ __forceinline__ double ce_gamma(const MaxwellCell &mc, const CeCell &m, const double xi[3])
{
    const double cx = xi[0] - mc.q[1], cy = xi[1] - mc.q[2], cz = xi[2] - mc.q[3];
    const double c2 = cx * cx + cy * cy + cz * cz;
    const double s = m.sxx * cx * cx + m.syy * (cy * cy + cz * cz) + 2.0 * (m.sxy * cx * cy + m.sxz * cx * cz);
    return 1.0 + s / (2.0 * m.prt) + (m.qx * cx / m.prt) * (c2 / (5.0 * m.RT) - 1.0);
}

// Velocities of an NS-corrected sample: attempt 0 uses the sample's own words w0 (velocities from
// w0[2..9], acceptance from w0[10..11]); attempt a > 0 draws the counters (id, 4j..4j+2, step,
// SAMPLE + 8a).  After kCeAttempts rejections the attempt-0 Maxwellian is kept.
__device__ __noinline__ void ce_xi(const InstDev &I, uint32_t id, uint32_t j, uint32_t step, const MaxwellCell &mc,
                                   const CeCell &ce, const uint32_t *w0, double xi[3])
{
    maxwell_xi(mc, w0 + 2, xi);
    if (u53(w0[10], w0[11]) * ce.A < ce_gamma(mc, ce, xi)) return;
    uint32_t w[12];
    double t[3];
    for (int a = 1; a < kCeAttempts; ++a) {
#pragma unroll
        for (uint32_t k = 0; k < 3; ++k) draw(I, id, 4u * j + k, step, kSample + 8u * static_cast<uint32_t>(a), w + 4 * k);
        maxwell_xi(mc, w + 2, t);
        if (u53(w[10], w[11]) * ce.A < ce_gamma(mc, ce, t)) {
            xi[0] = t[0]; xi[1] = t[1]; xi[2] = t[2];
            return;
        }
    }
}

// Single-precision rounding of the 53-bit uniform u53(a, b) (exact integer conversion, then a power
// of two): the same value as rounding the double u53(a, b).
__device__ __forceinline__ float u53_float(uint32_t a, uint32_t b)
{
    const unsigned long long m = (static_cast<unsigned long long>(a) << 21) | static_cast<unsigned long long>(b >> 11);
    return __ull2float_rn(m) * 0x1p-53f;
}

template <typename Rec, bool kRolled = true>
__device__ __forceinline__ Rec sample_particle(const InstDev &I, uint32_t id, uint32_t j, uint32_t step, const MaxwellCell &mc,
                                           const CeCell *ce)
{
    uint32_t w[12];
#pragma unroll
    for (uint32_t t = 0; t < 3; ++t) draw(I, id, 4u * j + t, step, kSample, w + 4 * t);
    Rec r;
    using T = decltype(r.xl);
    T x, xi[3];
    if (ce) {
        // NS-corrected option: the acceptance test needs the double-precision velocities
        x = (sizeof(T) == 4) ? static_cast<T>(u53_float(w[0], w[1])) : static_cast<T>(u53(w[0], w[1]));
        double xd[3];
        ce_xi(I, id, j, step, mc, *ce, w, xd);
#pragma unroll
        for (int d = 0; d < 3; ++d) xi[d] = store_val(xd[d], T());
    } else if constexpr (sizeof(T) == 4) {
        // single-precision records: double-single evaluation, double precision only where the
        // rounding of a component cannot be guaranteed
        x = u53_float(w[0], w[1]);
        if (!ds_maxwell<kRolled>(g_turn, g_logt, mc.U, mc.s, w + 2, xi)) {
            const float4 f = maxwell_fp64_from(I.R, mc.qp, make_uint4(w[2], w[3], w[4], w[5]),
                                               make_uint4(w[6], w[7], w[8], w[9]));
            xi[0] = f.y;
            xi[1] = f.z;
            xi[2] = f.w;
        }
    } else {
        x = u53(w[0], w[1]);
        maxwell_fp64<T>(mc, w + 2, xi);
    }
    if (x >= T(1)) x = sizeof(T) == 4 ? T(0x1.fffffep-1f) : x;
    r.xl = x;
    r.u = xi[0];
    r.v = xi[1];
    r.w = xi[2];
    return r;
}

// Samples j0..j1-1 of interior cell g (local index i) under the NS-corrected option, one per lane,
// into dst[j]: the per-cell factor once, then the samples (Maxwellian where the factor is off).
template <typename Rec>
__device__ __noinline__ void sample_run_ce(const InstDev &I, const double *prim, const int32_t *valid, int g, int i,
                                           uint32_t step, Rec *dst, int j0, int j1, int lane)
{
    const MaxwellCell mc = maxwell_cell(I, prim + 5 * g);
    CeCell ce;
    const bool on = ce_coefs(I, prim, valid, g, i, ce);
    for (int j = j0 + lane; j < j1; j += 32)
        st_rec(dst + j, sample_particle<Rec>(I, cell_id(I, i), static_cast<uint32_t>(j), step, mc, on ? &ce : nullptr));
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


// Majorant factor (c_max/c_ref)^{-2 upsilon} of the NTC count; kept per cell and recomputed only when
// c_max is raised.
__device__ __noinline__ double majorant_factor(const InstDev &I, double cmax)   // rare: when c_max rises
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
    // N and N - 1 converted by integer operations (exact)
    const double rr = (I.ntc_rate == 1) ? rho_t * I.inv_rho_ref : fixed_to_double(N, 0) * I.ntc_rr;
    const double nsel = I.ntc_A * rr * fixed_to_double(N - 1, 0) * fmaj * cmax;
    if (!dbl_lt(nsel, 1e8)) return -1;
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

// ------------------------------------------------------------------------------------------
// NTC collisions (Appendix A).  Candidates are taken in order in batches: a batch is cut before the
// first candidate that shares a particle with an earlier one in the batch, and after the first whose
// c_r raises c_max; inside such a prefix the candidates touch disjoint particles and see the same
// c_max, so doing them at once gives exactly the sequential result.
// ------------------------------------------------------------------------------------------

// Acceptance of a candidate: u < (c_r/c_max)^{1-2 upsilon} with u = u53(w2, w3).  Decided in single
// precision first: u lies in [uf, uf + 2^-24) with uf from the top 24 bits of w2, and for a ratio
// x32 = c_r/c_max above 1e-30 (relative speed above 1e-12) the single-precision power has a relative
// error below 1e-5; outside the margin 2e-4 p + 2.5e-7 around the threshold the decision is the exact
// one.  Inside it (and for tiny ratios) c_r and the power are evaluated in double precision.
// cr / exact: the exact relative speed, computed here when needed.
// The acceptance decided in double precision (the single-precision test was within its margin): out
// of line, as it is rare.  Records and results pass by value, so that no caller's record needs an
// address (a record whose address reaches a call lives in local memory on every path).
struct AcceptExact {
    double cr;     // the exact relative speed
    bool acc;
};
template <typename Rec>
__device__ __noinline__ AcceptExact accept_exact(const InstDev &I, double expo, Rec A, Rec B, double cm, uint32_t w2,
                                                 uint32_t w3, double cr, bool exact)
{
    if (!exact) cr = rel_speed(A, B);
    const double x = cr / cm;
    return AcceptExact{cr, u53(w2, w3) < ((I.upsilon == 0.0) ? x : pow(x, expo))};
}

template <typename Rec>
__device__ __forceinline__ bool accept_pair(const InstDev &I, double expo, float expo_f, const Rec &A, const Rec &B,
                                            float cr32, float cm32, double cm, uint32_t w2, uint32_t w3, double &cr,
                                            bool &exact)
{
    if (expo == 0.0) return true;                    // Maxwell molecules: every candidate collides
    const float x32 = cr32 / cm32;
    if (cr32 > 1e-12f && x32 > 1e-30f) {
        const float p32 = (I.upsilon == 0.0) ? x32 : exp2f(expo_f * log2f(x32));
        const float m32 = 2e-4f * p32 + 2.5e-7f;
        const float uf = static_cast<float>(w2 >> 8) * 0x1p-24f;
        if (uf < p32 - m32) return true;
        if (uf > p32 + m32) return false;
    }
    const AcceptExact r = accept_exact<Rec>(I, expo, A, B, cm, w2, w3, cr, exact);
    cr = r.cr;
    exact = true;
    return r.acc;
}

// Isotropic VHS scattering of an accepted pair (Appendix A) in double precision: the relative
// velocity keeps its magnitude c_r and takes the direction (theta, phi) with cos(theta) = 2 u1 - 1,
// phi = 2 pi u2 (u1 = u53(v0, v1), u2 = u53(v2, v3)).  Out of line, records by value.
template <typename Rec>
struct RecPair {
    Rec a, b;
};
template <typename Rec>
__device__ __noinline__ RecPair<Rec> scatter_fp64(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3, Rec A, Rec B,
                                                  double cr)
{
    using T = decltype(A.xl);
    const double ct = 2.0 * u53(v0, v1) - 1.0;
    const double st = sqrt(1.0 - ct * ct);
    double sp, cp;
    sincos(kTwoPi * u53(v2, v3), &sp, &cp);
    const double c0 = (cr * st) * cp, c1 = (cr * st) * sp, c2 = cr * ct;
    const double au = A.u, av = A.v, aw = A.w, bu = B.u, bv = B.v, bw = B.w;
    const double m0 = (au + bu) * 0.5, m1 = (av + bv) * 0.5, m2 = (aw + bw) * 0.5;
    A.u = store_val(m0 + c0 * 0.5, T());
    A.v = store_val(m1 + c1 * 0.5, T());
    A.w = store_val(m2 + c2 * 0.5, T());
    B.u = store_val(m0 - c0 * 0.5, T());
    B.v = store_val(m1 - c1 * 0.5, T());
    B.w = store_val(m2 - c2 * 0.5, T());
    return RecPair<Rec>{A, B};
}

// Scattering of accepted candidate k.  cr / exact: the double-precision relative speed when the
// caller already has it.  Single-precision records are scattered in double-single arithmetic, which
// yields the single-precision rounding of the same values as the double-precision evaluation; the
// few pairs where that cannot be guaranteed take the double-precision path.
__device__ __forceinline__ RecPair<RecD> scatter_pair(const InstDev &I, uint32_t id, uint32_t k, uint32_t step, RecD A,
                                                      RecD B, double cr, bool exact)
{
    uint32_t v[4];
    draw(I, id, 2u * k + 1u, step, kCollide, v);
    return scatter_fp64<RecD>(v[0], v[1], v[2], v[3], A, B, exact ? cr : rel_speed(A, B));
}
// (one copy, called from every collision loop: inlined five times it crowded the instruction cache)
__device__ __noinline__ RecPair<RecF> scatter_pair(const InstDev &I, uint32_t id, uint32_t k, uint32_t step, RecF A,
                                                   RecF B, double cr, bool exact)
{
    uint32_t v[4];
    draw(I, id, 2u * k + 1u, step, kCollide, v);
    float o[6];
    if (ds_scatter(g_turn, A.u, A.v, A.w, B.u, B.v, B.w, v[0], v[1], v[2], v[3], o)) {
        A.u = o[0]; A.v = o[1]; A.w = o[2];
        B.u = o[3]; B.v = o[4]; B.w = o[5];
        return RecPair<RecF>{A, B};
    }
    return scatter_fp64<RecF>(v[0], v[1], v[2], v[3], A, B, exact ? cr : rel_speed(A, B));
}

// The nc candidates of a staged cell list (nc from ntc_candidates), in order; candidate k is drawn
// in the batch that reaches it.
// A cell's particle list as collide_list sees it: position x -> record address.
template <typename Rec>
struct StagedList {
    Rec *p;
    __device__ __forceinline__ Rec *at(int x) const { return p + x; }
};

constexpr int kHash = 128;             // slots of a warp's touched-particle table (at most 2 x kMaxDirect keys)

// Slot of list position x in the slots [base, base + size) of the touched-particle table (inserted
// if absent; `fresh`: by this call).  At most size/2 keys share those slots, so a free slot or the
// key itself is always found within the probe limit.
__device__ __forceinline__ int seg_insert(int *key, int base, int size, int x, bool &fresh, int32_t *err)
{
    int h = base + static_cast<int>(__umulhi(static_cast<uint32_t>(x) * 2654435761u, static_cast<uint32_t>(size)));
    for (int it = 0; it < size; ++it) {
        const int old = atomicCAS(&key[h], -1, x);
        if (old == -1 || old == x) {
            fresh = (old == -1);
            return h;
        }
        h = (h + 1 == base + size) ? base : h + 1;
    }
    set_err(err, kErrOverflow);
    fresh = false;
    return base;
}

template <typename Rec>
struct CollideShared {
    int key[kHash];     // list position of the particle held in the slot, -1 = empty
    int own[kHash];     // lowest candidate of the current batch that touches the slot (32 = none)
    int mod[kHash];     // changed by an accepted collision
    Rec rec[kHash];
};

// Batches of up to 32 candidates cut before the first one that shares a particle with a
// lower lane's (found through a hash of the batch's picks: key, the list position; own, the lowest
// lane touching it; clear between batches) and after the first that raises c_max, the records read
// and written in place.
template <typename Rec, typename List>
__device__ __forceinline__ void collide_list_cut(const InstDev &I, uint32_t id, uint32_t step, List list, int N, int64_t nc,
                                                 double &cmax, int &nacc, int *s_key, int *s_own, int32_t *err)
{
    const int lane = threadIdx.x & 31;
    nacc = 0;
    if (N < 2 || nc <= 0) return;
    const double expo = 1.0 - 2.0 * I.upsilon;
    const float expo_f = static_cast<float>(expo);
    int acc = 0;
    double cm = cmax;
    for (int t = lane; t < kHash; t += 32) {
        s_key[t] = -1;
        s_own[t] = 32;
    }
    __syncwarp();
    for (int64_t k0 = 0; k0 < nc;) {
        const int64_t k = k0 + lane;
        const bool act = k < nc;
        uint32_t a = 0, b = 0, w2 = 0, w3 = 0;
        if (act) {
            uint32_t w[4];
            draw(I, id, static_cast<uint32_t>(2 * k), step, kCollide, w);
            a = idx32(w[0], static_cast<uint32_t>(N));
            b = idx32(w[1], static_cast<uint32_t>(N - 1));
            if (b >= a) ++b;
            w2 = w[2];
            w3 = w[3];
        }
        int ha = 0, hb = 0;
        if (act) {
            bool fresh;
            ha = seg_insert(s_key, 0, kHash, static_cast<int>(a), fresh, err);
            hb = seg_insert(s_key, 0, kHash, static_cast<int>(b), fresh, err);
            atomicMin(&s_own[ha], lane);
            atomicMin(&s_own[hb], lane);
        }
        __syncwarp();
        const bool conf = act && (s_own[ha] < lane || s_own[hb] < lane);
        const unsigned cmask = __ballot_sync(0xffffffffu, conf);
        const int navail = static_cast<int>(min(static_cast<int64_t>(32), nc - k0));
        const int m1 = cmask ? min(navail, __ffs(cmask) - 1) : navail;
        Rec A, B;
        float cr32 = 0.f;
        double cr = 0.0;
        bool exact = false;
        const float cm32 = static_cast<float>(cm);
        Rec *pA = nullptr, *pB = nullptr;
        if (lane < m1) {
            pA = list.at(static_cast<int>(a));
            pB = list.at(static_cast<int>(b));
            A = ld_rec_rw(pA);
            B = ld_rec_rw(pB);
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
            accd = (lane == fr) || accept_pair<Rec>(I, expo, expo_f, A, B, cr32, cm32, cm, w2, w3, cr, exact);
            if (accd) {
                const RecPair<Rec> r = scatter_pair(I, id, static_cast<uint32_t>(k), step, A, B, cr, exact);
                st_rec(pA, r.a);
                st_rec(pB, r.b);
            }
        }
        acc += __popc(__ballot_sync(0xffffffffu, accd));
        if (fr < m) cm = cr_r;
        __syncwarp();
        if (act) {
            s_key[ha] = -1;
            s_key[hb] = -1;
            s_own[ha] = 32;
            s_own[hb] = 32;
        }
        __syncwarp();
        k0 += m;
    }
    cmax = cm;
    nacc = acc;
}

// Dependency rounds: batches of up to 32 candidates on a warp, candidate k0 + lane on its lane.  The batch's particles
// are held in a shared-memory table (a hash of their list positions: key; the lowest remaining
// candidate touching each: own) and the candidates run in dependency rounds: a candidate runs once
// it is the lowest remaining candidate of the batch on both of its particles, so every particle sees
// its collisions in candidate order -- the sequential order of the NTC loop -- while independent
// candidates run together.  The changed records are written back after the batch.  Every candidate
// of a batch tests against the batch's c_max; where one raises it (Appendix A: c_max is raised to the
// pair's c_r before its test), the table is reloaded from memory and the batch rerun up to that
// candidate, and the next batch starts after it with the raised c_max.
template <typename Rec, typename List>
__device__ __forceinline__ void collide_list_rounds(const InstDev &I, uint32_t id, uint32_t step, List list, int N,
                                                    int64_t nc, double &cmax, int &nacc, CollideShared<Rec> &S,
                                                    int32_t *err)
{
    const int lane = threadIdx.x & 31;
    nacc = 0;
    if (N < 2 || nc <= 0) return;
    const double expo = 1.0 - 2.0 * I.upsilon;
    const float expo_f = static_cast<float>(expo);
    int acc = 0;
    double cm = cmax;
    for (int t = lane; t < kHash; t += 32) {
        S.key[t] = -1;
        S.own[t] = 32;
        S.mod[t] = 0;
    }
    __syncwarp();
    for (int64_t k0 = 0; k0 < nc;) {
        const int nb = static_cast<int>(min(static_cast<int64_t>(32), nc - k0));
        const int64_t k = k0 + lane;
        const bool act = lane < nb;
        uint32_t a = 0, b = 0, w2 = 0, w3 = 0;
        int ha = 0, hb = 0;
        bool fa = false, fb = false;
        if (act) {
            uint32_t w[4];
            draw(I, id, static_cast<uint32_t>(2 * k), step, kCollide, w);
            a = idx32(w[0], static_cast<uint32_t>(N));
            b = idx32(w[1], static_cast<uint32_t>(N - 1));
            if (b >= a) ++b;
            w2 = w[2];
            w3 = w[3];
            ha = seg_insert(S.key, 0, kHash, static_cast<int>(a), fa, err);
            hb = seg_insert(S.key, 0, kHash, static_cast<int>(b), fb, err);
        }
        // the rounds of candidates [0, limit) of the batch on the table; returns the accepted ones and
        // the lowest candidate that raised c_max (32: none) with its c_r
        auto rounds = [&](int limit, int &rmin, double &cr_r) -> int {
            if (fa) { S.rec[ha] = ld_rec_rw(list.at(static_cast<int>(a))); S.mod[ha] = 0; }
            if (fb) { S.rec[hb] = ld_rec_rw(list.at(static_cast<int>(b))); S.mod[hb] = 0; }
            __syncwarp();
            bool undone = lane < limit;
            int na = 0;
            rmin = 32;
            cr_r = 0.0;
            const float cm32 = static_cast<float>(cm);
            while (__any_sync(0xffffffffu, undone)) {
                if (undone) {
                    atomicMin(&S.own[ha], lane);
                    atomicMin(&S.own[hb], lane);
                }
                __syncwarp();
                const bool run = undone && S.own[ha] == lane && S.own[hb] == lane;
                __syncwarp();
                if (undone) {
                    S.own[ha] = 32;
                    S.own[hb] = 32;
                }
                bool accd = false, raises = false;
                double cr = 0.0;
                if (run) {
                    const Rec A = S.rec[ha], B = S.rec[hb];
                    const float cr32 = rel_speed_f32(A, B);
                    bool exact = false;
                    if (cr32 > cm32 * 0.99999f) {      // possibly above c_max: decide exactly
                        cr = rel_speed(A, B);
                        exact = true;
                    }
                    raises = exact && cr > cm;
                    accd = raises || accept_pair<Rec>(I, expo, expo_f, A, B, cr32, cm32, cm, w2, w3, cr, exact);
                    if (accd) {
                        const RecPair<Rec> r = scatter_pair(I, id, static_cast<uint32_t>(k), step, A, B, cr, exact);
                        S.rec[ha] = r.a;
                        S.rec[hb] = r.b;
                        S.mod[ha] = 1;
                        S.mod[hb] = 1;
                    }
                    undone = false;
                }
                const unsigned rm = __ballot_sync(0xffffffffu, raises);
                if (rm) {
                    const int r0 = __ffs(rm) - 1;
                    const double c0 = __shfl_sync(0xffffffffu, cr, r0);
                    if (r0 < rmin) {
                        rmin = r0;
                        cr_r = c0;
                    }
                }
                na += __popc(__ballot_sync(0xffffffffu, accd));
                __syncwarp();
            }
            return na;
        };
        __syncwarp();
        int rmin;
        double cr_r;
        int na = rounds(nb, rmin, cr_r);
        if (rmin < 32) {
            // candidates after the first raise saw the old c_max: rerun the batch up to it
            const int r_first = rmin;
            __syncwarp();
            na = rounds(r_first + 1, rmin, cr_r);
            if (rmin != r_first) set_err(err, kErrOverflow);   // (cannot happen: same inputs)
        }
        __syncwarp();
        if (fa && S.mod[ha]) st_rec(list.at(static_cast<int>(a)), S.rec[ha]);
        if (fb && S.mod[hb]) st_rec(list.at(static_cast<int>(b)), S.rec[hb]);
        __syncwarp();
        if (act) {
            S.key[ha] = -1;
            S.key[hb] = -1;
            S.mod[ha] = 0;
            S.mod[hb] = 0;
        }
        __syncwarp();
        acc += na;
        if (rmin < 32) {
            cm = cr_r;
            k0 += rmin + 1;
        } else {
            k0 += nb;
        }
    }
    cmax = cm;
    nacc = acc;
}

// The nc NTC candidates of a cell's list of N records in candidate order (one warp).  A staged list
// (the survivors of the absorption and the re-sampled particles of a P > 0 cell, up to kRoundsMaxN
// records) has many candidates sharing a particle within a batch of 32: the dependency rounds keep
// the batches whole (the Sod Kn sweep: 0.40 -> 0.33 ms per step).  The direct cells' lists (P = 0)
// take the cut batches, measured faster there (the shock batch: 0.912 vs 0.920 ms per step).
constexpr int kRoundsMaxN = 1024;

template <typename Rec, typename List>
__device__ __noinline__ void collide_list(const InstDev &I, uint32_t id, uint32_t step, List list, int N, int64_t nc,
                                          double &cmax, int &nacc, CollideShared<Rec> &S, int32_t *err)
{
    constexpr bool staged = std::is_same<List, StagedList<Rec>>::value;
    if (staged && N <= kRoundsMaxN)
        collide_list_rounds<Rec>(I, id, step, list, N, nc, cmax, nacc, S, err);
    else collide_list_cut<Rec>(I, id, step, list, N, nc, cmax, nacc, S.key, S.own, err);
}

// ------------------------------------------------------------------------------------------
// Exact fixed-point sums of particle moments: velocities at 2^-40, |xi|^2/2 at 2^-32.  Integer
// sums do not depend on the order of accumulation, so the per-cell flux sums are identical for
// every launch shape, and the global particle-flux ledger telescopes exactly.
// ------------------------------------------------------------------------------------------
// x * 2^S rounded to the nearest integer (ties to even): the product by the power of two is exact,
// then one conversion; |x| must stay below 2^(62-S) (guarded by the caller's range check).
template <int S>
__device__ __forceinline__ long long fx_bits(float x)
{
    return __float2ll_rn(__fmul_rn(x, static_cast<float>(1ull << S)));
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

// Prefetch of the 128-byte line holding p into L2 (a hint: no register, no fault on any address).
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" :: "l"(p));
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

// Address of position x of a cell's arrived (sorted) list: far movers from the left, the left
// neighbour's R run (stored backwards), the cell's S run, the right neighbour's L run, far movers
// from the right.
template <typename Rec, typename FR>
__device__ __forceinline__ Rec *arrived_ptr(int x, const CellHdr &h, Rec *in, FR *fs)
{
    int r = x;
    if (r < h.nfb) return &fs[h.fb + r].rec;
    r -= h.nfb;
    if (r < h.Rn) return in + (h.Rend - 1 - r);
    r -= h.Rn;
    if (r < h.Sn) return in + (h.Sa + r);
    r -= h.Sn;
    if (r < h.Ln) return in + (h.La + r);
    r -= h.Ln;
    return &fs[h.fb + h.nfb + r].rec;
}

// Record x of a direct cell's list after re-sampling: the arrived positions, then the re-sampled
// particles after them in the cell's output block blk.
template <typename Rec, typename FR>
__device__ __forceinline__ Rec *list_rec(int x, const CellHdr &h, Rec *in, FR *fs, Rec *blk)
{
    return x < h.n_in ? arrived_ptr<Rec>(x, h, in, fs) : blk + x;
}

// Whether a direct cell's re-sampled particles (if any) are in place before the collision kernels
// run: none, or all drawn ahead by k_sample (kPreSampleMin or more of them).
__device__ __forceinline__ bool light_resampling(const CellHdr &h)
{
    return h.n_new == 0 || h.n_new >= kPreSampleMin;
}

// ------------------------------------------------------------------------------------------
// Collision kernel.  Runs before the streaming kernel on the cells of class kClsDirect and
// kClsStaged (work list built by k_offsets_flux):
//   direct: the candidate pairs depend only on counters, so up to 32 of them are drawn at once;
//           the touched particles (at most 64) are loaded into a shared-memory table keyed by list
//           position, collided there in candidate order, and the changed ones written back in
//           place, into the arrived runs or the far-mover list, where the streaming kernel reads
//           them; cells with more candidates or with re-sampled particles (drawn first, after the
//           arrived positions) run the candidates in batches on that list in place;
//   staged: the survivors of the absorption draw (Eq. p) and the re-sampled particles (Eq.
//           maxsample) are written to the first half of the cell's output block and collided there;
//           the streaming kernel reads this list instead of the arrived runs.
// ------------------------------------------------------------------------------------------
constexpr int kCollideThreads = 128;

// Position of the n-th (from 0) set bit of m (m has more than n set bits).
__device__ __forceinline__ int nth_set_bit(unsigned m, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Light direct cells (P = 0, 1..kMaxDirect candidates, nothing re-sampled or every re-sampled particle
// drawn ahead by k_sample, as in a first step), packed: the warp holds
// the cells of list positions t0..n_items-1 (at most 32; one round of pack_rounds) and runs them in
// rounds.  A round takes the next cells whose candidates fit in the 32 lanes together:
// cell c on lanes [b_c, b_c + nc_c), lane b_c + k its candidate k, with the table slots
// [4 b_c, 4 (b_c + nc_c)) to itself.  Each ballot is masked
// to the cell's lanes, so every cell follows exactly the batches of a cell alone: its candidates
// drawn at once (the pairs depend only on counters), a batch cut before the first candidate that
// shares a particle with an earlier one of the batch and after the first whose c_r raises c_max.
// The touched particles are loaded into the table by the lane that inserted them, collided there
// in candidate order and the changed ones written back in place (into the arrived runs, the
// far-mover list or the re-sampled positions of the output block, where the streaming kernel reads
// them).
template <typename Rec>
__device__ __forceinline__ void collide_packed(const EngineDev &E, const int32_t *list, int t0, int n_items,
                                               CollideShared<Rec> &S, Rec *in, Rec *out, FarItem<Rec> *fs)
{
    const int lane = threadIdx.x & 31;
    const unsigned upto = 0xffffffffu >> (31 - lane);          // lanes 0..lane
    int cg = -1, cn = 0;                                        // the chunk's cell at this lane
    if (t0 + lane < n_items) {
        cg = list[t0 + lane];
        const CellHdr *hp = E.hdr + cg;
        const int nc = hp->nc;
        if (hp->cls == kClsDirect && light_resampling(*hp) && nc >= 1 && nc <= kMaxDirect) cn = nc;
    }
    int done = 0;                                               // chunk cells collided so far
    while (__any_sync(0xffffffffu, lane >= done && cn > 0)) {
        int x = (lane >= done) ? cn : 0;                        // inclusive candidate count
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const bool inr = lane >= done && x <= 32;
        const unsigned rm = __ballot_sync(0xffffffffu, inr);
        const unsigned cells = __ballot_sync(0xffffffffu, inr && cn > 0);
        const unsigned starts = __reduce_or_sync(0xffffffffu, (inr && cn > 0) ? (1u << (x - cn)) : 0u);
        const int last = 31 - __clz(rm);
        const int total = __shfl_sync(0xffffffffu, x, last);
        done = last + 1;
        // this lane's cell and candidate
        const bool act = lane < total;
        const int sb = act ? 31 - __clz(starts & upto) : 0;
        const int src = act ? nth_set_bit(cells, __popc(starts & upto) - 1) : 0;
        const int g = __shfl_sync(0xffffffffu, cg, src);
        const int cn_src = __shfl_sync(0xffffffffu, cn, src);
        const int nc = act ? cn_src : 0;
        const int kc = lane - sb;
        if (act && !(kc >= 0 && kc < nc && sb + nc <= 32)) set_err(E.err, kErrOverflow);   // (cannot happen)
        const unsigned segmask = act ? ((0xffffffffu >> (32 - nc)) << sb) : 0u;
        for (int t = lane; t < 4 * total; t += 32) {
            S.key[t] = -1;
            S.own[t] = 32;
            S.mod[t] = 0;
        }
        __syncwarp();
        const CellHdr *hp = E.hdr + (act ? g : 0);
        const InstDev &I = E.inst[act ? hp->b : 0];
        int sa = 0, sc = 0;
        bool fa = false, fb = false;
        uint32_t w2 = 0, w3 = 0;
        Rec *blk = nullptr;
        if (act) {
            const int N = hp->n_in + hp->n_new;
            blk = out + hp->off;
            uint32_t w[4];
            draw(I, cell_id(I, hp->i), 2u * static_cast<uint32_t>(kc), I.step, kCollide, w);
            const int pa = static_cast<int>(idx32(w[0], static_cast<uint32_t>(N)));
            int pb = static_cast<int>(idx32(w[1], static_cast<uint32_t>(N - 1)));
            if (pb >= pa) ++pb;
            w2 = w[2];
            w3 = w[3];
            sa = seg_insert(S.key, 4 * sb, 4 * nc, pa, fa, E.err);
            sc = seg_insert(S.key, 4 * sb, 4 * nc, pb, fb, E.err);
            if (fa) S.rec[sa] = ld_rec_rw(list_rec<Rec>(pa, *hp, in, fs, blk));
            if (fb) S.rec[sc] = ld_rec_rw(list_rec<Rec>(pb, *hp, in, fs, blk));
        }
        __syncwarp();
        double cm = act ? E.cmax[g] : 0.0;
        int acc = 0, k0 = 0;
        bool raised = false;
        while (__any_sync(0xffffffffu, k0 < nc)) {
            const bool live = act && kc >= k0;
            if (live) { atomicMin(&S.own[sa], kc); atomicMin(&S.own[sc], kc); }
            __syncwarp();
            const bool conf = live && (S.own[sa] < kc || S.own[sc] < kc);
            const unsigned cmask = (__ballot_sync(0xffffffffu, conf) & segmask) >> sb;
            const int end1 = cmask ? __ffs(cmask) - 1 : nc;     // first candidate that shares a particle
            const bool inb = live && kc < end1;
            Rec A, B;
            float cr32 = 0.f;
            double cr = 0.0;
            bool exact = false;
            const float cm32 = static_cast<float>(cm);
            if (inb) {
                A = S.rec[sa];
                B = S.rec[sc];
                cr32 = rel_speed_f32(A, B);
                if (cr32 > cm32 * 0.99999f) {      // possibly above c_max: decide exactly
                    cr = rel_speed(A, B);
                    exact = true;
                }
            }
            const unsigned rmask = (__ballot_sync(0xffffffffu, inb && exact && cr > cm) & segmask) >> sb;
            const int fr = rmask ? __ffs(rmask) - 1 : 32;
            const int end = min(end1, fr + 1);
            const double cr_r = __shfl_sync(0xffffffffu, cr, sb + (fr < 32 ? fr : 0));
            bool accd = false;
            if (live && kc < end) {
                accd = (kc == fr) || accept_pair<Rec>(I, I.vhs_expo, I.vhs_expo_f, A, B, cr32, cm32, cm, w2, w3, cr, exact);
                if (accd) {
                    const RecPair<Rec> r = scatter_pair(I, cell_id(I, hp->i), static_cast<uint32_t>(kc), I.step, A, B,
                                                        cr, exact);
                    S.rec[sa] = r.a;
                    S.rec[sc] = r.b;
                    S.mod[sa] = 1;
                    S.mod[sc] = 1;
                }
            }
            acc += __popc(__ballot_sync(0xffffffffu, accd) & segmask);
            if (fr < end) {
                cm = cr_r;
                raised = true;
            }
            __syncwarp();
            if (live) { S.own[sa] = 32; S.own[sc] = 32; }
            __syncwarp();
            if (k0 < nc) k0 = end;
        }
        if (act) {
            if (fa && S.mod[sa]) st_rec(list_rec<Rec>(S.key[sa], *hp, in, fs, blk), S.rec[sa]);
            if (fb && S.mod[sc]) st_rec(list_rec<Rec>(S.key[sc], *hp, in, fs, blk), S.rec[sc]);
            if (kc == 0) {
                E.ncand[g] = nc;
                E.nacc[g] = acc;
                if (raised) {
                    E.cmax[g] = cm;
                    E.fmaj[g] = majorant_factor(I, cm);
                }
            }
        }
        __syncwarp();
    }
}

// The list of a direct cell, read and updated in place: the arrived positions, then the re-sampled
// particles after them in the cell's output block.
template <typename Rec>
struct ArrivedList {
    const CellHdr *h;
    Rec *in;
    FarItem<Rec> *fs;
    Rec *blk;
    __device__ __forceinline__ Rec *at(int x) const { return x < h->n_in ? arrived_ptr<Rec>(x, *h, in, fs) : blk + x; }
};

// Direct cells with more than kMaxDirect candidates or with re-sampled particles, one per warp: the
// re-sampled particles first (sampling precedes the collisions), written after the arrived positions
// in the output block; then the candidates in batches of up to 32 (cut at the first pair that shares
// a particle with an earlier one of the batch), the records read and written in place, where the
// streaming kernel reads them.
template <typename Rec>
__device__ __noinline__ void collide_big(const EngineDev &E, int g, CollideShared<Rec> &S, Rec *in, Rec *out,
                                         FarItem<Rec> *fs)
{
    const int lane = threadIdx.x & 31;
    const CellHdr *hp = E.hdr + g;
    const InstDev &I = E.inst[hp->b];
    const int nc = hp->nc, n_in = hp->n_in, nn = hp->n_new, i = hp->i;
    const uint32_t id = cell_id(I, i), step = I.step;
    Rec *blk = out + hp->off;
    if (nn > 0 && !(hp->edges & kEdgePresampled)) {       // (otherwise drawn ahead by k_sample)
        if (I.resample_mode == 1) {
            sample_run_ce<Rec>(I, E.prim, E.valid, g, i, step, blk + n_in, 0, nn, lane);
        } else {
            const MaxwellCell mc = maxwell_cell_for<Rec>(I, E.prim + 5 * g);
            for (int j = lane; j < nn; j += 32)
                st_rec(blk + n_in + j, sample_particle<Rec>(I, id, static_cast<uint32_t>(j), step, mc, nullptr));
        }
        __syncwarp();
    }
    const double cm0 = E.cmax[g];
    double cmax = cm0;
    int na = 0;
    collide_list<Rec>(I, id, step, ArrivedList<Rec>{hp, in, fs, blk}, n_in + nn, nc, cmax, na, S, E.err);
    if (lane == 0) {
        E.ncand[g] = nc;
        E.nacc[g] = na;
        if (cmax != cm0) {
            E.cmax[g] = cmax;
            E.fmaj[g] = majorant_factor(I, cmax);
        }
    }
}

// Absorption draw u53(w0, w1) < P decided on the first word: with T = floor(P 2^32), w0 < T means
// u < P and w0 > T means u >= P; only w0 = T needs the 53-bit value.
__device__ __forceinline__ bool absorbed(uint32_t w0, uint32_t w1, double P, uint32_t T, bool all)
{
    if (all) return true;
    if (w0 != T) return w0 < T;
    return u53(w0, w1) < P;
}

template <typename Rec>
__device__ __noinline__ void collide_staged(const EngineDev &E, const InstDev &I, const CellHdr &h, int g, CollideShared<Rec> &S,
                               Rec *in, Rec *out, FarItem<Rec> *fs)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t id = cell_id(I, h.i), step = I.step;
    const double P = E.P[g];
    const bool all = !(P < 1.0);                       // u53 < 1 always
    const uint32_t T = all ? 0u : static_cast<uint32_t>(floor(P * 4294967296.0));
    Rec *stage = out + h.off;
    int run = 0;
    for (int base = 0; base < h.n_in; base += 32) {
        const int k = base + lane;
        Rec v;
        bool keep = false;
        if (k < h.n_in) {
            v = ld_rec_rw(arrived_ptr<Rec>(k, h, in, fs));
            keep = true;
            if (P > 0.0) {
                uint32_t w[4];
                draw(I, id, static_cast<uint32_t>(k), step, kAbsorb, w);
                keep = !absorbed(w[0], w[1], P, T, all);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) st_rec(stage + run + __popc(m & lt), v);
        run += __popc(m);
    }
    const double rho_t = E.psi[5 * g];
    const double rho_w = rho_t - static_cast<double>(run) * I.mp_over_dx;
    const int64_t nn = E.valid[g] ? resample_count(I, id, step, P, rho_w) : 0;
    const int64_t n_tot = run + nn;
    if (n_tot > h.slots) {
        if (lane == 0) {
            set_err(E.err, kErrOverflow);
            E.hdr[g].cls = kClsSkip;
        }
        return;
    }
    if (nn > 0) {
        if (I.resample_mode == 1) {
            sample_run_ce<Rec>(I, E.prim, E.valid, g, h.i, step, stage + run, 0, static_cast<int>(nn), lane);
        } else {
            const MaxwellCell mc = maxwell_cell_for<Rec>(I, E.prim + 5 * g);
            for (int j = lane; j < nn; j += 32)
                st_rec(stage + run + j, sample_particle<Rec>(I, id, static_cast<uint32_t>(j), step, mc, nullptr));
        }
    }
    __syncwarp();
    const double cm0 = E.cmax[g];
    double cmax = cm0;
    int64_t nc = ntc_candidates(I, id, step, static_cast<int>(n_tot), rho_t, cmax, E.fmaj[g]);
    if (nc < 0) {
        if (lane == 0) set_err(E.err, kErrOverflow);
        nc = 0;
    }
    int na = 0;
    collide_list<Rec>(I, id, step, StagedList<Rec>{stage}, static_cast<int>(n_tot), nc, cmax, na, S, E.err);
    if (lane == 0) {
        E.ncand[g] = static_cast<int32_t>(nc);
        E.nacc[g] = na;
        E.nabs[g] = h.n_in - run;
        E.nnew[g] = static_cast<int32_t>(nn);
        if (cmax != cm0) {
            E.cmax[g] = cmax;
            E.fmaj[g] = majorant_factor(I, cmax);
        }
    }
}


// ------------------------------------------------------------------------------------------
// Block kernel k_cellblock: one block of kBlockThreads per cell, persistent blocks over the work list
// of the cells with many collision candidates (the heavy list: staged cells, P > 0, and direct cells,
// P = 0, whose candidate count is at least kHeavyCandidates; the lighter ones run one warp per cell
// in the collision kernel).  Step 2 of Sec. 3.4 in the order the paper gives it:
//   absorption (staged cells): particle k of the arrived list is absorbed into the wave with
//     probability P (Eq. p); the survivors keep their order, compacted by the whole block into the
//     first half of the cell's output block;
//   re-sampling: (1-P) of the wave (Eq. maxsample), after the survivors (staged) or after the
//     arrived positions in the output block (direct), by the whole block;
//   NTC collisions (Appendix A) on that list.  Candidate k touches particles a_k, b_k and must see
//     them as every earlier candidate left them; candidates are taken in windows of kWindow and
//     executed in rounds: a candidate runs in the first round in which no earlier unfinished
//     candidate of the window touches either of its particles (each round every unfinished candidate
//     claims its two particles with atomicMax of (round, -position); the lowest position wins, so the
//     earliest unfinished candidate always runs and a window needs at most kWindow rounds).  The
//     candidates that may run in a round are packed into the first threads of the block, so that
//     only as many warps as there are runnable candidates / 32 execute the scattering.  This is the
//     sequential result whenever c_max stays fixed.  A candidate whose c_r exceeds c_max raises it,
//     and every later candidate must use the raised value: the window is first run with the
//     window's c_max; if any candidate raised it, the records are put back as they were at the
//     window's start and only the candidates up to the first raising one are run again (the raising
//     one accepted, as the sequential loop accepts it), and the next window starts after it with the
//     raised c_max.
// The records live in a shared-memory table during the collisions: the whole list when it has at
// most kBlockSlots records (slot = list position), otherwise the particles a window of kWindowHashed
// candidates touches (hashed by list position); the changed records are written back after each
// window.
// ------------------------------------------------------------------------------------------
constexpr int kBlockThreads = 128;
constexpr int kPer = 2;                             // window candidates per thread (window 256: the
                                                    // smaller tables fit five blocks per SM)
constexpr int kWindow = kPer * kBlockThreads;       // candidates per window (table = the whole list)
constexpr int kWindowHashed = kBlockThreads * 2;    // candidates per window when the touched particles are hashed
constexpr int kBlockSlots = 1024;      // table slots (the hashed form holds at most 2 x kWindowHashed keys)
static_assert((kBlockSlots & (kBlockSlots - 1)) == 0 && 4 * kWindowHashed <= kBlockSlots,
              "hashed table: a power of two, at most half full");
static_assert(kWindowHashed <= kWindow, "the window arrays hold a hashed window");
constexpr int kAbsorbPer = 4;          // arrived records per thread in flight in the absorption pass
constexpr int kHeavyCandidates = 96;   // candidates from which a cell takes the block kernel

template <typename Rec>
struct BlockShared {
    int key[kBlockSlots];          // hashed form: list position held by the slot, -1 = empty
    unsigned own[kBlockSlots];     // claim of the current round: (round << 16) | (0xffff - window position)
    unsigned char mod[kBlockSlots];// changed in the current window
    Rec rec[kBlockSlots];          // current values
    int2 ab[kWindow];              // table slots of each candidate's pair
    uint2 wa[kWindow];             // acceptance draw
    float4 sc[kWindow][2];         // scattering: the angle parts (single-precision records) or the draw
    unsigned char acc[kWindow];    // accepted
    unsigned char angok[kWindow];  // the angle parts are usable
    short ready[kWindow];          // the candidates that run in the current round
    CellHdr hdr;
    MaxwellCell mc;                // the cell's sampling state
    CeCell ce;
    int ce_on;
    int wsum[kAbsorbPer][kBlockThreads / 32];
    int item, nn, nc, ok, rmin, nready[2];     // nready: the round's list length, by round parity
    double cm_new;
};

__device__ __forceinline__ int block_insert(int *key, int x, int32_t *err)
{
    uint32_t h = __umulhi(static_cast<uint32_t>(x) * 2654435761u, static_cast<uint32_t>(kBlockSlots));
    for (int it = 0; it < kBlockSlots; ++it) {
        const int old = atomicCAS(&key[h], -1, x);
        if (old == -1 || old == x) return static_cast<int>(h);
        h = (h + 1u) & (kBlockSlots - 1);
    }
    set_err(err, kErrOverflow);
    return 0;
}

// What the acceptance test of a window needs, formed once per window.  The single-precision ratio
// c_r / c_max is taken as c_r * (1 / c_max): within two units in the last place of the quotient,
// far inside the margin outside of which the single-precision decision is the exact one (the margin
// covers a 1e-5 relative error of the single-precision power).
struct WindowConst {
    double cm, expo;
    float cm32, cm32_near, inv_cm32, expo_f;
    bool always, linear;     // Maxwell molecules (exponent 0); hard spheres (exponent 1)
};

// Candidate c of the window run on the current records.  id, k0: the cell's generator id and the
// window's first candidate (for the draw of a pair that needs the double-precision scattering).
template <typename Rec>
__device__ __forceinline__ void block_run_candidate(const InstDev &I, BlockShared<Rec> &S, int c, const WindowConst &W,
                                                    bool redo, uint32_t id, uint32_t step, int64_t k0)
{
    const int sa = S.ab[c].x, sb = S.ab[c].y;
    Rec A = S.rec[sa], B = S.rec[sb];
    const float cr32 = rel_speed_f32(A, B);
    double cr = 0.0;
    bool exact = false;
    if (cr32 > W.cm32_near) {          // possibly above c_max: decide exactly
        cr = rel_speed(A, B);
        exact = true;
    }
    bool a;
    const uint32_t w2 = S.wa[c].x, w3 = S.wa[c].y;
    if (exact && cr > W.cm) {          // c_max raised to c_r: accepted
        a = true;
        atomicMin(&S.rmin, c);
        if (redo) S.cm_new = cr;       // in the rerun only the first raising candidate runs
    } else if (W.always) {
        a = true;
    } else {
        const float x32 = cr32 * W.inv_cm32;
        bool decided = false;
        a = false;
        if (cr32 > 1e-12f && x32 > 1e-30f) {
            const float p32 = W.linear ? x32 : exp2f(W.expo_f * log2f(x32));
            const float m32 = 2e-4f * p32 + 2.5e-7f;
            const float uf = static_cast<float>(w2 >> 8) * 0x1p-24f;
            if (uf < p32 - m32) { a = true; decided = true; }
            else if (uf > p32 + m32) decided = true;
        }
        if (!decided) {
            const AcceptExact r = accept_exact<Rec>(I, W.expo, A, B, W.cm, w2, w3, cr, exact);
            cr = r.cr;
            exact = true;
            a = r.acc;
        }
    }
    if (a) {
        bool done = false;
        if constexpr (sizeof(A.u) == 4) {
            if (S.angok[c]) {
                const float4 g0 = S.sc[c][0], g1 = S.sc[c][1];
                const DsAngles g{{g0.x, g0.y}, {g0.z, g0.w}, {g1.x, g1.y}, {g1.z, g1.w}};
                float o[6];
                if (ds_scatter_apply(A.u, A.v, A.w, B.u, B.v, B.w, g, o)) {
                    A.u = o[0]; A.v = o[1]; A.w = o[2];
                    B.u = o[3]; B.v = o[4]; B.w = o[5];
                    done = true;
                }
            }
            if (!done) {
                uint32_t v[4];
                draw(I, id, static_cast<uint32_t>(2 * (k0 + c) + 1), step, kCollide, v);
                const RecPair<Rec> r = scatter_fp64<Rec>(v[0], v[1], v[2], v[3], A, B, exact ? cr : rel_speed(A, B));
                A = r.a;
                B = r.b;
            }
        } else {
            const float4 g0 = S.sc[c][0];
            const RecPair<Rec> r = scatter_fp64<Rec>(__float_as_uint(g0.x), __float_as_uint(g0.y), __float_as_uint(g0.z),
                                                     __float_as_uint(g0.w), A, B, exact ? cr : rel_speed(A, B));
            A = r.a;
            B = r.b;
        }
        S.rec[sa] = A;
        S.rec[sb] = B;
        S.mod[sa] = 1;
        S.mod[sb] = 1;
    }
    S.acc[c] = a ? 1 : 0;
}

// One pass of rounds over the window's candidates c < live_end.  Returns when all have run.
template <typename Rec>
__device__ void block_rounds(const InstDev &I, BlockShared<Rec> &S, int live_end, const WindowConst &W, bool redo,
                             uint32_t id, uint32_t step, int64_t k0)
{
    const int t = threadIdx.x, lane = t & 31;
    const unsigned lt = (1u << lane) - 1u;
    bool undone[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) undone[u] = t + u * kBlockThreads < live_end;
    // each round: the ready check of the claims made before it, a barrier, then the runs beside
    // the claims of the next round (the runs touch the records, the claims only own), a barrier
    auto claim = [&](unsigned round) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int c = t + u * kBlockThreads;
            if (undone[u]) {
                const unsigned code = (round << 16) | (0xffffu - static_cast<unsigned>(c));
                atomicMax(&S.own[S.ab[c].x], code);
                atomicMax(&S.own[S.ab[c].y], code);
            }
        }
    };
    claim(1u);
    if (t == 0) {
        S.nready[0] = 0;
        S.nready[1] = 0;
    }
    __syncthreads();
    int remaining = live_end;
    for (unsigned round = 1; round <= kWindow + 1 && remaining > 0; ++round) {
        const int par = static_cast<int>(round & 1u);
        // the runnable candidates, appended to the round's list (any order: they touch disjoint particles)
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int c = t + u * kBlockThreads;
            const unsigned code = (round << 16) | (0xffffu - static_cast<unsigned>(c));
            const bool rdy = undone[u] && S.own[S.ab[c].x] == code && S.own[S.ab[c].y] == code;
            const unsigned m = __ballot_sync(0xffffffffu, rdy);
            if (m) {
                int pos = 0;
                if (lane == __ffs(m) - 1) pos = atomicAdd(&S.nready[par], __popc(m));
                pos = __shfl_sync(0xffffffffu, pos, __ffs(m) - 1);
                if (rdy) {
                    S.ready[pos + __popc(m & lt)] = static_cast<short>(c);
                    undone[u] = false;
                }
            }
        }
        __syncthreads();
        const int total = S.nready[par];
        if (t == 0) S.nready[par ^ 1] = 0;          // the next round's list (last read a round ago)
        for (int j = t; j < total; j += kBlockThreads)
            block_run_candidate<Rec>(I, S, S.ready[j], W, redo, id, step, k0);
        claim(round + 1u);
        remaining -= total;
        __syncthreads();
    }
}

// The list of a staged cell (its output block) and of a direct cell (the arrived positions, then the
// re-sampled particles after them in the output block), position -> record address.
template <typename Rec>
struct BlockList {
    const CellHdr *h;       // in shared memory
    Rec *in;
    FarItem<Rec> *fs;
    Rec *blk;
    bool staged;
    __device__ __forceinline__ Rec *at(int x) const
    {
        if (staged || x >= h->n_in) return blk + x;
        return arrived_ptr<Rec>(x, *h, in, fs);
    }
};

// The nc candidates of a list of N records (written earlier by this block or in place).  The list
// in memory holds the state at the start of each window: the changed records are written back after
// every window, and a window rerun after a raise of c_max reloads them from there.
template <typename Rec>
__device__ void block_collisions(const EngineDev &E, const InstDev &I, uint32_t id, uint32_t step,
                                 const BlockList<Rec> &L, int N, int64_t nc, BlockShared<Rec> &S, double &cmax,
                                 int &nacc)
{
    const int t = threadIdx.x;
    const double expo = 1.0 - 2.0 * I.upsilon;
    const bool whole = N <= kBlockSlots;          // the whole list in the table, slot = position
    const int win = whole ? kWindow : kWindowHashed;
    double cm = cmax;
    int na = 0;
    if (N < 2 || nc <= 0) {
        nacc = 0;
        return;
    }
    if (whole) {
        for (int x = t; x < N; x += kBlockThreads) {
            S.rec[x] = ld_rec_rw(L.at(x));
            S.mod[x] = 0;
        }
    }
    int64_t k_lo = 0;
    while (k_lo < nc) {
        const int nw = static_cast<int>(min(static_cast<int64_t>(win), nc - k_lo));
        if (whole) {
            for (int x = t; x < N; x += kBlockThreads) S.own[x] = 0u;
        } else {
            for (int x = t; x < kBlockSlots; x += kBlockThreads) { S.key[x] = -1; S.own[x] = 0u; S.mod[x] = 0; }
        }
        if (t == 0) S.rmin = kWindow;
        __syncthreads();
        for (int c = t; c < nw; c += kBlockThreads) {
            const int64_t k = k_lo + c;
            uint32_t w[4], v[4];
            draw(I, id, static_cast<uint32_t>(2 * k), step, kCollide, w);
            const int a = static_cast<int>(idx32(w[0], static_cast<uint32_t>(N)));
            int b = static_cast<int>(idx32(w[1], static_cast<uint32_t>(N - 1)));
            if (b >= a) ++b;
            draw(I, id, static_cast<uint32_t>(2 * k + 1), step, kCollide, v);
            S.wa[c] = make_uint2(w[2], w[3]);
            if constexpr (sizeof(Rec().u) == 4) {
                // the scattering angles depend only on the draw: formed here for every candidate at once
                DsAngles g;
                const bool ok = ds_scatter_angles(g_turn, v[0], v[1], v[2], v[3], g);
                S.angok[c] = ok ? 1 : 0;
                S.sc[c][0] = make_float4(g.ct.hi, g.ct.lo, g.st.hi, g.st.lo);
                S.sc[c][1] = make_float4(g.cp.hi, g.cp.lo, g.sp.hi, g.sp.lo);
            } else {
                S.sc[c][0] = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]),
                                         __uint_as_float(v[3]));
            }
            if (whole) S.ab[c] = make_int2(a, b);
            else S.ab[c] = make_int2(block_insert(S.key, a, E.err), block_insert(S.key, b, E.err));
        }
        if (!whole) {
            __syncthreads();
            for (int x = t; x < kBlockSlots; x += kBlockThreads) {
                const int y = S.key[x];
                if (y >= 0) S.rec[x] = ld_rec_rw(L.at(y));
            }
        }
        __syncthreads();
        WindowConst W;
        W.cm = cm;
        W.expo = expo;
        W.cm32 = static_cast<float>(cm);
        W.cm32_near = W.cm32 * 0.99999f;
        W.inv_cm32 = 1.0f / W.cm32;
        W.expo_f = static_cast<float>(expo);
        W.always = (expo == 0.0);
        W.linear = (I.upsilon == 0.0);
        block_rounds<Rec>(I, S, nw, W, false, id, step, k_lo);
        const int r = S.rmin;
        int upto = nw;
        if (r < nw) {
            // the candidates after position r saw c_max before its raise: back to the window's start
            // (the records in memory) and again up to r only
            const int n_slots = whole ? N : kBlockSlots;
            for (int x = t; x < n_slots; x += kBlockThreads) {
                if (S.mod[x]) S.rec[x] = ld_rec_rw(L.at(whole ? x : S.key[x]));
                S.mod[x] = 0;
                S.own[x] = 0u;
            }
            __syncthreads();
            block_rounds<Rec>(I, S, r + 1, W, true, id, step, k_lo);
            cm = S.cm_new;
            upto = r + 1;
        }
        int mine = 0;
        for (int c = t; c < upto; c += kBlockThreads) mine += S.acc[c];
        na += __syncthreads_count(mine == 1) + 2 * __syncthreads_count(mine == 2) +
              3 * __syncthreads_count(mine == 3) + 4 * __syncthreads_count(mine == 4);
        const int n_slots = whole ? N : kBlockSlots;
        for (int x = t; x < n_slots; x += kBlockThreads) {
            if (S.mod[x]) {
                st_rec(L.at(whole ? x : S.key[x]), S.rec[x]);
                S.mod[x] = 0;
            }
        }
        __syncthreads();
        k_lo += upto;
    }
    cmax = cm;
    nacc = na;
}

// Staged cell: absorption and compaction of the survivors into the first half of the output block.
// Returns the survivors.
template <typename Rec>
__device__ int block_absorb(const EngineDev &E, const InstDev &I, const CellHdr &h, int g, BlockShared<Rec> &S,
                            Rec *in, FarItem<Rec> *fs, Rec *stage, uint32_t id, uint32_t step)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const double P = E.P[g];
    const bool all = !(P < 1.0);                       // u53 < 1 always
    const uint32_t T = all ? 0u : static_cast<uint32_t>(floor(P * 4294967296.0));
    int run = 0;
    for (int base = 0; base < h.n_in; base += kAbsorbPer * kBlockThreads) {
        Rec v[kAbsorbPer];
        bool keep[kAbsorbPer];
#pragma unroll
        for (int u = 0; u < kAbsorbPer; ++u) {
            const int k = base + u * kBlockThreads + t;
            keep[u] = k < h.n_in;
            if (keep[u]) v[u] = ld_rec_rw(arrived_ptr<Rec>(k, h, in, fs));
        }
#pragma unroll
        for (int u = 0; u < kAbsorbPer; ++u) {
            const int k = base + u * kBlockThreads + t;
            if (keep[u] && P > 0.0) {
                uint32_t w[4];
                draw(I, id, static_cast<uint32_t>(k), step, kAbsorb, w);
                keep[u] = !absorbed(w[0], w[1], P, T, all);
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep[u]);
            if (lane == 0) S.wsum[u][warp] = __popc(m);
        }
        __syncthreads();
        int pre = run;
#pragma unroll
        for (int u = 0; u < kAbsorbPer; ++u) {
            int before = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < kBlockThreads / 32; ++w) {
                const int c = S.wsum[u][w];
                before += (w < warp) ? c : 0;
                tot += c;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep[u]);
            if (keep[u]) st_rec(stage + pre + before + __popc(m & lt), v[u]);
            pre += tot;
        }
        run = pre;
        __syncthreads();
    }
    return run;
}

template <typename Rec>
__device__ void block_cell(const EngineDev &E, int g, BlockShared<Rec> &S, Rec *in, Rec *out, FarItem<Rec> *fs)
{
    const int t = threadIdx.x;
    if (t == 0) S.hdr = E.hdr[g];
    __syncthreads();
    const CellHdr &h = S.hdr;
    const InstDev &I = E.inst[h.b];
    const bool staged = h.cls == kClsStaged;
    const uint32_t id = cell_id(I, h.i), step = I.step;
    Rec *blk = out + h.off;
    // the cell's sampling state, by one thread of the last warp while the others absorb
    if (t == kBlockThreads - 32 && (!staged || E.valid[g]) && (staged || h.n_new > 0)) {
        S.mc = maxwell_cell(I, E.prim + 5 * g);
        S.ce_on = (I.resample_mode == 1) ? (ce_coefs(I, E.prim, E.valid, g, h.i, S.ce) ? 1 : 0) : 0;
    }
    int run = h.n_in;
    if (staged) run = block_absorb<Rec>(E, I, h, g, S, in, fs, blk, id, step);
    // re-sampled and candidate counts
    if (t == 0) {
        if (staged) {
            const double rho_t = E.psi[5 * g];
            const double rho_w = rho_t - static_cast<double>(run) * I.mp_over_dx;
            const int64_t nn = E.valid[g] ? resample_count(I, id, step, E.P[g], rho_w) : 0;
            const int64_t n_tot = run + nn;
            S.ok = (n_tot <= h.slots) ? 1 : 0;
            S.nn = static_cast<int>(nn < h.slots ? nn : h.slots);
            int64_t nc = 0;
            if (S.ok) {
                nc = ntc_candidates(I, id, step, static_cast<int>(n_tot), rho_t, E.cmax[g], E.fmaj[g]);
                if (nc < 0 || nc > INT32_MAX) {
                    set_err(E.err, kErrOverflow);
                    nc = 0;
                }
            } else {
                set_err(E.err, kErrOverflow);
                E.hdr[g].cls = kClsSkip;
            }
            S.nc = static_cast<int>(nc);
        } else {
            S.ok = 1;
            S.nn = h.n_new;
            S.nc = h.nc;
        }
    }
    __syncthreads();
    if (!S.ok) return;
    const int nn = S.nn;
    const int n_tot = run + nn;
    if (nn > 0 && (staged || !(h.edges & kEdgePresampled))) {   // (otherwise drawn ahead by k_sample)
        const MaxwellCell mc = S.mc;
        const CeCell *ce = S.ce_on ? &S.ce : nullptr;
        for (int j = t; j < nn; j += kBlockThreads)
            st_rec(blk + run + j, sample_particle<Rec>(I, id, static_cast<uint32_t>(j), step, mc, ce));
    }
    __syncthreads();
    const double cm0 = E.cmax[g];
    double cmax = cm0;
    int na = 0;
    const BlockList<Rec> L{&S.hdr, in, fs, blk, staged};
    block_collisions<Rec>(E, I, id, step, L, n_tot, S.nc, S, cmax, na);
    if (t == 0) {
        E.ncand[g] = S.nc;
        E.nacc[g] = na;
        if (staged) {
            E.nabs[g] = h.n_in - run;
            E.nnew[g] = nn;
        }
        if (cmax != cm0) {
            E.cmax[g] = cmax;
            E.fmaj[g] = majorant_factor(I, cmax);
        }
    }
}

template <typename Rec, int kMinB>
__global__ void __launch_bounds__(kBlockThreads, kMinB) k_cellblock(const __grid_constant__ EngineDev E, int rp)
{
    wait_predecessor();
    extern __shared__ __align__(16) unsigned char smraw[];
    BlockShared<Rec> &S = *reinterpret_cast<BlockShared<Rec> *>(smraw);
    Rec *in = static_cast<Rec *>(E.buf[rp]);
    Rec *out = static_cast<Rec *>(E.buf[1 - rp]);
    FarItem<Rec> *fs = static_cast<FarItem<Rec> *>(E.far_sorted);
    const int n_items = E.ticket[kListLen + kHeavyList];
    if (n_items == 0) return;                 // (written by the kernel before: the same for every thread)
    const int32_t *list = E.wl + static_cast<size_t>(kHeavyList) * E.G;
    for (;;) {
        if (threadIdx.x == 0) S.item = atomicAdd(&E.ticket[kHeavyList], 1);
        __syncthreads();
        const int it = S.item;
        __syncthreads();
        if (it >= n_items) break;
        const int g = list[it];
        const int cls = E.hdr[g].cls;
        if (cls == kClsStaged || cls == kClsDirect) block_cell<Rec>(E, g, S, in, out, fs);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Particles drawn ahead (Eq. maxsample, or its NS-corrected option): the re-sampled particles of
// direct cells with at least kPreSampleMin of them -- every particle of a first step -- in chunks of
// kSampleChunk over all warps of the GPU, into the positions after the cell's arrived list in its
// output block, before the collision kernels collide them there.  First the rounds of the light list.
// ------------------------------------------------------------------------------------------
constexpr int kSampleThreads = 256;

// Rounds of the light list (one item each for the collision kernel): the light cells of each warp of
// k_offsets_flux (consecutive in the list), in order, in groups whose candidates fit in the 32
// lanes of a warp; one descriptor (first position, cells) per round.
// Returns the number of rounds; lane r < (that number) holds round r in `mine`.
__device__ __forceinline__ int pack_rounds(const EngineDev &E, int grp, int lane, int2 &mine)
{
    mine = make_int2(0, 0);
    const int n_groups = (E.G_run + 31) / 32;
    const int2 gr = (grp < n_groups) ? E.wgrp[grp] : make_int2(0, 0);
    if (gr.y <= 0) return 0;
    int ncl = 0;
    if (lane < gr.y) ncl = E.wlnc[gr.x + lane];
    int done = 0, nr = 0;
    while (__any_sync(0xffffffffu, lane >= done && ncl > 0)) {
        int x = (lane >= done) ? ncl : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const unsigned rm = __ballot_sync(0xffffffffu, lane >= done && x <= 32);
        const int last = min(31 - __clz(rm), gr.y - 1);
        if (lane == nr) mine = make_int2(gr.x + done, last + 1 - done);
        ++nr;
        done = last + 1;
    }
    return nr;
}

template <typename Rec>
__global__ void __launch_bounds__(kSampleThreads, 4) k_sample(const __grid_constant__ EngineDev E, int rp)
{
    wait_predecessor();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kW = kSampleThreads / 32;
    const int n_groups = (E.G_run + 31) / 32;
    // one group per warp, one atomic per block for the rounds of its warps
    __shared__ int s_nr[kW], s_base;
    for (int w0 = blockIdx.x * kW; w0 < n_groups; w0 += gridDim.x * kW) {
        int2 mine;
        const int nr = pack_rounds(E, w0 + warp, lane, mine);
        if (lane == 0) s_nr[warp] = nr;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < kW; ++k) tot += s_nr[k];
            s_base = tot ? atomicAdd(&E.ticket[kRoundLen], tot) : 0;
        }
        __syncthreads();
        int base = s_base;
        for (int k = 0; k < warp; ++k) base += s_nr[k];
        if (lane < nr) {
            if (base + lane < E.G) E.wr[base + lane] = mine;
            else set_err(E.err, kErrOverflow);
        }
        __syncthreads();
    }
    Rec *out = static_cast<Rec *>(E.buf[1 - rp]);
    const int n_chunks = min(E.ticket[kPreLen], E.wls_cap);
    if (n_chunks == 0) return;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&E.ticket[kPreCtr], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_chunks) break;
        const int2 it = E.wlp[t];
        const int g = it.x, j0 = it.y;
        const CellHdr &h = E.hdr[g];
        const int b = h.b, n_in = h.n_in, n_new = h.n_new, cls = h.cls, i = h.i;
        const long long off = h.off;
        if (cls != kClsDirect && cls != kClsStream) continue;
        const InstDev &I = E.inst[b];
        const int j1 = min(j0 + kSampleChunk, n_new);
        if (I.resample_mode == 1) {
            sample_run_ce<Rec>(I, E.prim, E.valid, g, i, I.step, out + off + n_in, j0, j1, lane);
            continue;
        }
        // (the draws unrolled here: this kernel's loop is short)
        const MaxwellCell mc = maxwell_cell_for<Rec>(I, E.prim + 5 * g);
        for (int j = j0 + lane; j < j1; j += 32)
            st_rec(out + off + n_in + j, sample_particle<Rec, false>(I, cell_id(I, i), static_cast<uint32_t>(j),
                                                                     I.step, mc, nullptr));
    }
}

template <typename Rec>
__global__ void __launch_bounds__(kCollideThreads, 8) k_collide(const __grid_constant__ EngineDev E, int rp)
{
    wait_predecessor();
    extern __shared__ __align__(16) unsigned char smraw[];
    CollideShared<Rec> &S = reinterpret_cast<CollideShared<Rec> *>(smraw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    Rec *in = static_cast<Rec *>(E.buf[rp]);
    Rec *out = static_cast<Rec *>(E.buf[1 - rp]);
    FarItem<Rec> *fs = static_cast<FarItem<Rec> *>(E.far_sorted);
    // the other cells of this kernel (direct cells with more than kMaxDirect candidates or with
    // re-sampled particles, staged cells), one per warp, then the rounds of the light direct cells
    // (packed by k_sample: one round is one item); the next ticket is fetched while the current item
    // runs (the heavy cells: k_cellblock)
    {
        const int n_items = E.ticket[kListLen + kWarpList];
        const int32_t *list = E.wl + static_cast<size_t>(kWarpList) * E.G;
        int t = 0;
        if (lane == 0) t = atomicAdd(&E.ticket[kWarpList], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        while (t < n_items) {
            int tn = 0;
            if (lane == 0) tn = atomicAdd(&E.ticket[kWarpList], 1);
            const int g = list[t];
            const CellHdr h = E.hdr[g];
            if (h.cls == kClsStaged) collide_staged<Rec>(E, E.inst[h.b], h, g, S, in, out, fs);
            else if (h.cls == kClsDirect) collide_big<Rec>(E, g, S, in, out, fs);
            __syncwarp();
            t = __shfl_sync(0xffffffffu, tn, 0);
        }
    }
    {
        const int n_rounds = min(E.ticket[kRoundLen], E.G);
        const int32_t *list = E.wl + static_cast<size_t>(kLightList) * E.G;
        const int n_light = E.ticket[kListLen + kLightList];
        int t = 0;
        if (lane == 0) t = atomicAdd(&E.ticket[kRoundCtr], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        while (t < n_rounds) {
            int tn = 0;
            if (lane == 0) tn = atomicAdd(&E.ticket[kRoundCtr], 1);
            const int2 r = E.wr[t];
            collide_packed<Rec>(E, list, r.x, min(r.x + min(r.y, 32), n_light), S, in, out, fs);
            t = __shfl_sync(0xffffffffu, tn, 0);
        }
    }
    // re-sampled particles of cells without collisions (Eq. maxsample), chunk by chunk, into the
    // positions after the cell's arrived list in its output block
    const int n_chunks = min(E.ticket[kSampleLen], E.wls_cap);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&E.ticket[kSampleCtr], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_chunks) break;
        const int2 it = E.wls[t];
        const int g = it.x, j0 = it.y;
        const CellHdr &h = E.hdr[g];
        const int b = h.b, n_in = h.n_in, n_new = h.n_new, cls = h.cls, i = h.i;
        const long long off = h.off;
        if (cls != kClsStream && cls != kClsReservoir) continue;
        const InstDev &I = E.inst[b];
        const int j1 = min(j0 + kSampleChunk, n_new);
        if (I.resample_mode == 1 && cls == kClsStream) {
            sample_run_ce<Rec>(I, E.prim, E.valid, g, i, I.step, out + off + n_in, j0, j1, lane);
            continue;
        }
        const MaxwellCell mc = maxwell_cell_for<Rec>(I, E.prim + 5 * g);
        for (int j = j0 + lane; j < j1; j += 32)
            st_rec(out + off + n_in + j, sample_particle<Rec>(I, cell_id(I, i), static_cast<uint32_t>(j), I.step, mc,
                                                              nullptr));
    }
}

// ------------------------------------------------------------------------------------------
// Streaming kernel: one warp per cell.
//
// Output block of a cell s (2 x slots records, slots = the bound on its list after re-sampling):
// particles that stay (S) are written forward from the block start, those moving one cell left
// (L) forward from the middle, those moving one cell right (R) backward from the end; each run
// keeps the order the particles had before transport.  The sorted list of cell g for the next
// step reads R(g-1) from its end backwards, then S(g), then L(g+1).  A staged cell's list lies
// in the first half of its own block; its stayers are written back in place, never ahead of the
// read position.  Any split of the list into consecutive groups gives the same stable order, so
// every piece of the list is streamed in its own groups of 32.
//
// Register use decides the bandwidth of this kernel (it needs about 48 resident warps per SM to
// keep HBM busy), so the loop state is small: the piece descriptors live in shared memory and the
// rare cases (walls, wraps, leavers, moves of two or more cells) share one code path.
// ------------------------------------------------------------------------------------------
// One piece of a cell's list: list positions [k0, k0 + n); kind 0: records at p[dir * r], read-only
// loads (arrived runs); 1: records at p[r], plain loads (records written by the collision kernel
// into the output block); 2: the records of the sorted far-list items p[r].
template <typename Rec>
struct Piece {
    const void *p;
    int n, k0, dir, kind;
};

template <typename Rec>
struct StreamShared {
    long long acc[4][32];     // lane-private rare-path sums (u, v, w, |xi|^2/2)
    Piece<Rec> piece[6];
};

// Records of the list in flight: kStreamStages iterations of 32 x groups records, each slot written
// (by an asynchronous copy) and read by the same lane.
constexpr int kStreamStages = 3;
template <typename Rec, int kGroups>
struct StreamRing {
    Rec rec[kStreamStages][32 * kGroups];
};

// Asynchronous 16-byte copy global -> shared (L2 only), its commit and the wait for all but the N
// most recent groups of this thread.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Address of position r of a piece of the list (kind 0: arrived runs, stored forward or backward;
// 1: records in the output block; 2: sorted far-list items).
template <typename Rec>
__device__ __forceinline__ const Rec *piece_rec(const Piece<Rec> &pc, int r)
{
    if (pc.kind == 2) return &static_cast<const FarItem<Rec> *>(pc.p)[r].rec;
    return static_cast<const Rec *>(pc.p) + (pc.kind == 0 ? pc.dir * r : r);
}

struct StreamState {
    int oS, oL, oR;                       // next write offsets in the block: S, L (forward), R (backward)
    int ngone;                            // far movers and removed particles of this lane
    bool range_ok;
};

// Full transport of one particle (Step 3) with 64-bit cell arithmetic and the boundary conditions.
__device__ __forceinline__ int64_t transport_full(const InstDev &I, int64_t cell, float &xl, float &u, bool &refl)
{
    const float s = __fmaf_rn(u, I.dtdx_f, xl);
    if (!(fabsf(s) < 1e15f)) return kGone;
    const float fk = floorf(s);
    float x = __fsub_rn(s, fk);
    int64_t k = static_cast<int64_t>(fk);
    if (x >= 1.0f) { x = 0.0f; k += 1; }
    xl = x;
    return apply_walls<float>(I, cell + k, xl, u, refl);
}
__device__ __forceinline__ int64_t transport_full(const InstDev &I, int64_t cell, double &xl, double &u, bool &refl)
{
    return transport(I, cell, xl, u, refl);
}

// Everything but a move to the same or a neighbouring cell inside the domain: wall reflections,
// periodic wraps, particles that leave the domain or move two or more cells.  The particle is
// transported from its original state with the boundary conditions; particles that move two or
// more cells or leave take their pre-transport moments out of the cell (a far mover is appended to
// the far list), a reflected particle's normal momentum changes sign (+2 u after the reflection).
// Returns the class: 0 one cell left, 1 stays, 2 one cell right, 3 farther, 4 left the domain.
template <typename Rec>
__device__ __forceinline__ int stream_rare(const EngineDev &E, int g, int k, Rec &v, long long *a, StreamState &st)
{
    using T = decltype(Rec().xl);
    const CellHdr &h = E.hdr[g];
    const InstDev &I = E.inst[h.b];
    const int ci = h.i;
    const T u0 = v.u;
    bool refl = false;
    const int64_t d = transport_full(I, ci, v.xl, v.u, refl);
    int c;
    if (d == kGone) c = 4;
    else if (d == ci) c = 1;
    else if (d == ci - 1) c = 0;
    else if (d == ci + 1) c = 2;
    else c = 3;
    if (refl || c >= 3) {
        st.range_ok = st.range_ok && fx_in_range(u0) && fx_in_range(v.v) && fx_in_range(v.w);
        if (c >= 3) {
            ++st.ngone;
            a[0] -= fx_vel(u0);
            a[32] -= fx_vel(v.v);
            a[64] -= fx_vel(v.w);
            a[96] -= fx_energy(u0, v.v, v.w);
        } else {
            a[0] += fx_vel(v.u) - fx_vel(u0);
        }
        if (c == 3) {
            const int slot = atomicAdd(&E.far_count[0], 1);
            if (slot < E.far_cap) {
                FarItem<Rec> it;
                it.dest = I.cell_base + 1 + static_cast<int>(d);
                it.src = g;
                it.q = k;
                it.pad = 0;
                it.rec = v;
                static_cast<FarItem<Rec> *>(E.far_app)[slot] = it;
            } else {
                set_err(E.err, kErrOverflow);
            }
        }
    }
    return c;
}

// Common path of the transport: c in {0, 1, 2} for the same or a neighbouring cell inside the
// cells [lo, lo + width) (the domain, and the phantom cell beyond an end that faces another part of
// a split domain); 4 for a particle of an inflow/outflow reservoir (ci = -1 or C) that stays outside
// the domain on the reservoir's side (discarded: a reservoir keeps only what enters, and its own
// moment sums are not used); -1 for everything else (general path).
__device__ __forceinline__ int move_near(float dtdx, int C, int lo, int width, int ci, float &xl, float u)
{
    const float s = __fmaf_rn(u, dtdx, xl);
    if (!(fabsf(s) < 1073741824.0f)) return -1;
    const float fk = floorf(s);
    float x = __fsub_rn(s, fk);
    int k = __float2int_rz(fk);                  // |fk| <= 2^30: exact
    if (x >= 1.0f) { x = 0.0f; k += 1; }
    const unsigned dd = static_cast<unsigned>(k + 1);
    const int d = ci + k;                        // |ci| <= 2^30, |k| <= 2^30: no overflow
    if (dd >= 3u || static_cast<unsigned>(d - lo) >= static_cast<unsigned>(width)) {
        if ((d < 0 && ci < 0) || (d >= C && ci >= C)) return 4;
        return -1;
    }
    xl = x;
    return static_cast<int>(dd);
}
__device__ __forceinline__ int move_near(double dtdx, int C, int lo, int width, int ci, double &xl, double u)
{
    const double s = __fma_rn(u, dtdx, xl);
    if (!(fabs(s) < 1073741824.0)) return -1;
    const double fk = floor(s);
    double x = __dsub_rn(s, fk);
    int k = __double2int_rz(fk);
    if (x >= 1.0) { x = 0.0; k += 1; }
    const unsigned dd = static_cast<unsigned>(k + 1);
    const int d = ci + k;
    if (dd >= 3u || static_cast<unsigned>(d - lo) >= static_cast<unsigned>(width)) {
        if ((d < 0 && ci < 0) || (d >= C && ci >= C)) return 4;
        return -1;
    }
    xl = x;
    return static_cast<int>(dd);
}

// Moment sums of the L run (pL, nL) and the R run (pR, nR) of a block, read back together: the runs
// are taken as one list, two records per lane in flight per iteration.
template <typename Rec>
__device__ __forceinline__ void run_sums_lr(const Rec *pL, int nL, const Rec *pR, int nR, long long sL[4],
                                            long long sR[4], bool &ok)
{
    const int n = nL + nR;
    for (int j = threadIdx.x & 31; j < n; j += 64) {
        const int j2 = j + 32;
        const Rec a = ld_rec_rw(j < nL ? pL + j : pR + (j - nL));
        Rec b = a;
        if (j2 < n) b = ld_rec_rw(j2 < nL ? pL + j2 : pR + (j2 - nL));
        const long long fa[4] = {fx_vel(a.u), fx_vel(a.v), fx_vel(a.w), fx_energy(a.u, a.v, a.w)};
        ok = ok && fx_in_range(a.u) && fx_in_range(a.v) && fx_in_range(a.w);
        const bool aL = j < nL;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sL[k] += aL ? fa[k] : 0;
            sR[k] += aL ? 0 : fa[k];
        }
        if (j2 < n) {
            const long long fb[4] = {fx_vel(b.u), fx_vel(b.v), fx_vel(b.w), fx_energy(b.u, b.v, b.w)};
            ok = ok && fx_in_range(b.u) && fx_in_range(b.v) && fx_in_range(b.w);
            const bool bL = j2 < nL;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                sL[k] += bL ? fb[k] : 0;
                sR[k] += bL ? 0 : fb[k];
            }
        }
    }
}

// Warp sum of a 64-bit integer whose lane values stay below 2^62 in magnitude: three 32-bit
// reductions of its 21-bit limbs (the limb sums of 32 lanes fit in 32 bits).
__device__ __forceinline__ long long warp_sum_ll(long long x)
{
    const unsigned a0 = static_cast<unsigned>(x) & 0x1fffffu;
    const unsigned a1 = static_cast<unsigned>(x >> 21) & 0x1fffffu;
    const int a2 = static_cast<int>(x >> 42);
    const unsigned s0 = __reduce_add_sync(0xffffffffu, a0);
    const unsigned s1 = __reduce_add_sync(0xffffffffu, a1);
    const int s2 = __reduce_add_sync(0xffffffffu, a2);
    return static_cast<long long>(s2) * (1LL << 42) + static_cast<long long>(s1) * (1LL << 21) + static_cast<long long>(s0);
}

// Outputs of a cell that streams nothing (skipped, or in error).
__device__ __forceinline__ void stream_cell_empty(const EngineDev &E, int g, int wp)
{
    const int lane = threadIdx.x & 31;
    if (lane < 4) { E.AL[4 * g + lane] = 0; E.AR[4 * g + lane] = 0; }
    if (lane < 5) E.Aself[5 * g + lane] = 0;
    if (lane == 0) {
        E.nL[wp][g] = 0; E.nS[wp][g] = 0; E.nR[wp][g] = 0; E.slotsb[wp][g] = 0;
        E.ncand[g] = 0; E.nacc[g] = 0; E.nabs[g] = 0; E.nnew[g] = 0;
    }
}


// kMinBlocks: 512-thread blocks per SM the register budget allows; kStreamGroups: groups of 32 records
// each lane loads before any of them is processed (loads in flight per warp).  Both are launch knobs
// of the autotuner; results do not depend on them.
template <typename Rec, int kMinBlocks, int kStreamGroups>
__global__ void __launch_bounds__(512, kMinBlocks) k_stream(EngineDev E, int rp)
{
    wait_predecessor();
    using T = decltype(Rec().xl);
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * (blockDim.x >> 5) + warp;
    if (g >= E.G_run) return;
    StreamShared<Rec> &SS = reinterpret_cast<StreamShared<Rec> *>(s_raw)[warp];
    const int wp = 1 - rp;
    const CellHdr *hp = E.hdr + g;
    const int cls = hp->cls;
    int n_tot = 0;
    if (cls == kClsStaged) n_tot = hp->n_in - E.nabs[g] + E.nnew[g];
    else if (cls != kClsSkip) n_tot = hp->n_in + hp->n_new;
    const int slots = hp->slots;
    if (cls == kClsSkip || n_tot > slots) {
        if (cls != kClsSkip && lane == 0) set_err(E.err, kErrOverflow);
        stream_cell_empty(E, g, wp);
        return;
    }
    Rec *blk = static_cast<Rec *>(E.buf[wp]) + hp->off;
    // pieces of the list, in list order
    if (lane == 0) {
        const Rec *in = static_cast<const Rec *>(E.buf[rp]);
        const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
        if (cls == kClsStaged) {
            for (int q = 0; q < 5; ++q) SS.piece[q] = Piece<Rec>{blk, 0, 0, 1, 1};
            SS.piece[5] = Piece<Rec>{blk, n_tot, 0, 1, 1};
        } else {
            int k = 0;
            SS.piece[0] = Piece<Rec>{fs + hp->fb, hp->nfb, k, 1, 2};
            k += hp->nfb;
            SS.piece[1] = Piece<Rec>{in + (hp->Rend - 1), hp->Rn, k, -1, 0};
            k += hp->Rn;
            SS.piece[2] = Piece<Rec>{in + hp->Sa, hp->Sn, k, 1, 0};
            k += hp->Sn;
            SS.piece[3] = Piece<Rec>{in + hp->La, hp->Ln, k, 1, 0};
            k += hp->Ln;
            SS.piece[4] = Piece<Rec>{fs + hp->fb + hp->nfb, hp->nfa, k, 1, 2};
            k += hp->nfa;
            // re-sampled particles, drawn by the collision kernel after the arrived positions (the
            // stayers written so far lie below the read position)
            SS.piece[5] = Piece<Rec>{blk + k, n_tot - k, k, 1, 1};
        }
    }
    long long *acc = &SS.acc[0][lane];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[32 * j] = 0;
    __syncwarp();
    T dtdx;
    if constexpr (sizeof(T) == 4) dtdx = hp->dtdx_f;
    else dtdx = E.inst[hp->b].dtdx;
    const int C = hp->C, ci = hp->i;
    const int lo = -(hp->edges & 1), width = C + (hp->edges & 1) + ((hp->edges >> 1) & 1);
    const unsigned lt = (1u << lane) - 1u;
    StreamState st;
    st.oS = 0;
    st.oL = slots;
    st.oR = 2 * slots - 1;
    st.ngone = 0;
    st.range_ok = true;
    // The list, iteration by iteration (32 x groups positions of one piece each): the records of
    // the iteration kStreamStages - 1 ahead are copied into the warp's ring asynchronously while the
    // current one is transported, so the loads' latency is not waited for.
    StreamRing<Rec, kStreamGroups> &RG =
        reinterpret_cast<StreamRing<Rec, kStreamGroups> *>(s_raw + (blockDim.x >> 5) * sizeof(StreamShared<Rec>))[warp];
    constexpr int kIt = 32 * kStreamGroups;
    int qp = 0, bp = 0, sp = 0;                  // producer: piece, offset, stage
    while (qp < 6 && SS.piece[qp].n == 0) ++qp;
    int qc = qp, bc = 0, sc = 0;                 // consumer
    auto issue = [&]() {
        if (qp < 6) {
            const Piece<Rec> pc = SS.piece[qp];
#pragma unroll
            for (int u2 = 0; u2 < kStreamGroups; ++u2) {
                const int r = bp + 32 * u2 + lane;
                if (r < pc.n) {
                    const Rec *src = piece_rec(pc, r);
                    Rec *dst = &RG.rec[sp][32 * u2 + lane];
#pragma unroll
                    for (int h = 0; h < static_cast<int>(sizeof(Rec) / 16); ++h)
                        cp_async16(reinterpret_cast<char *>(dst) + 16 * h, reinterpret_cast<const char *>(src) + 16 * h);
                }
            }
            bp += kIt;
            if (bp >= pc.n) {
                bp = 0;
                do { ++qp; } while (qp < 6 && SS.piece[qp].n == 0);
            }
        }
        cp_async_commit();                        // (an empty group past the end keeps the count aligned)
        sp = (sp + 1 == kStreamStages) ? 0 : sp + 1;
    };
#pragma unroll
    for (int s0 = 0; s0 < kStreamStages - 1; ++s0) issue();
    while (qc < 6) {
        issue();
        cp_async_wait<kStreamStages - 1>();       // this iteration's copies (each lane reads its own)
        const int n = SS.piece[qc].n, k0 = SS.piece[qc].k0;
        const int base = bc;
#pragma unroll
        for (int u2 = 0; u2 < kStreamGroups; ++u2) {
            const int r = base + 32 * u2 + lane;
            if (base + 32 * u2 >= n) break;
            Rec v;
            int c = 5;
            if (r < n) {
                v = RG.rec[sc][32 * u2 + lane];
                c = move_near(dtdx, C, lo, width, ci, v.xl, v.u);
                if (c < 0) c = stream_rare<Rec>(E, g, k0 + r, v, acc, st);
            }
            const unsigned mL = __ballot_sync(0xffffffffu, c == 0);
            const unsigned mS = __ballot_sync(0xffffffffu, c == 1);
            const unsigned mR = __ballot_sync(0xffffffffu, c == 2);
            const unsigned m = (c == 0) ? mL : ((c == 1) ? mS : mR);
            const int rk = __popc(m & lt);
            const int o = (c == 0) ? st.oL + rk : ((c == 1) ? st.oS + rk : st.oR - rk);
            if (c < 3) st_rec(blk + o, v);
            st.oS += __popc(mS);
            st.oL += __popc(mL);
            st.oR -= __popc(mR);
        }
        bc += kIt;
        if (bc >= n) {
            bc = 0;
            do { ++qc; } while (qc < 6 && SS.piece[qc].n == 0);
        }
        sc = (sc + 1 == kStreamStages) ? 0 : sc + 1;
    }
    cp_async_wait<0>();
    __syncwarp();
    // moments of the L and R runs, read back with every lane busy
    const int nLr = st.oL - slots;
    const int nRr = 2 * slots - 1 - st.oR;
    long long sL[4] = {0, 0, 0, 0}, sR[4] = {0, 0, 0, 0};
    bool ok = st.range_ok;
    run_sums_lr<Rec>(blk + slots, nLr, blk + st.oR + 1, nRr, sL, sR, ok);
    if (!__all_sync(0xffffffffu, ok) && lane == 0) set_err(E.err, kErrOverflow);
    long long lj = 0, rj = 0, gj = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const long long a = warp_sum_ll(sL[j]), b = warp_sum_ll(sR[j]), c = warp_sum_ll(acc[32 * j]);
        if (lane == j) { lj = a; rj = b; gj = c; }
    }
    const int ngone = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(st.ngone));
    if (lane < 4) {
        E.AL[4 * g + lane] = lj;
        E.AR[4 * g + lane] = rj;
        E.Aself[5 * g + 1 + lane] = gj - lj - rj;
    }
    if (lane == 0) {
        E.Aself[5 * g] = -static_cast<int64_t>(ngone + nLr + nRr);
        E.nS[wp][g] = st.oS;
        E.nL[wp][g] = nLr;
        E.nR[wp][g] = nRr;
        E.slotsb[wp][g] = slots;
        if (cls != kClsStaged) {
            if (cls != kClsDirect) { E.ncand[g] = 0; E.nacc[g] = 0; }
            E.nabs[g] = 0;
            E.nnew[g] = hp->n_new;
        }
        if (cls != kClsReservoir) atomicAdd(&E.inst[hp->b].updates, static_cast<unsigned long long>(n_tot));
    }
}

// ------------------------------------------------------------------------------------------
// Far movers: rank sort by (dest, src, q) -- keys are unique.
// ------------------------------------------------------------------------------------------
template <typename Rec>
__global__ void k_far_sort(EngineDev E)
{
    wait_predecessor();
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

// s = a + b as 64-bit integers; false when the sum overflows.
__device__ __forceinline__ bool add_no_overflow(long long a, long long b, long long &s)
{
    s = static_cast<long long>(static_cast<unsigned long long>(a) + static_cast<unsigned long long>(b));
    return ((a ^ s) & (b ^ s)) >= 0;
}

// ------------------------------------------------------------------------------------------
// Cell kernel: Eq. (r1) update, time average, primitive state, P, slot bound and plan of the next
// step.  For P = 0 the re-sampled count and the NTC candidate count depend only on cell data and
// counters, so they are decided here, one thread per cell, instead of inside the particle kernels.
// ------------------------------------------------------------------------------------------
template <typename Rec, int B>
__global__ void __launch_bounds__(B) k_cells(EngineDev E, int q, int update)
{
    wait_predecessor();
    __shared__ int64_t s_w[B / 32];
    const int g = blockIdx.x * B + threadIdx.x;
    int64_t myslots = 0;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (update) E.far_count[0] = 0;
        for (int q = 0; q < kLists; ++q) E.ticket[kListLen + q] = 0;
        E.ticket[kSampleLen] = 0;
        E.ticket[kPreLen] = 0;
        E.ticket[kRoundLen] = 0;
    }
    if (g < E.G_run) {
        CellHdr hd;
        hd.Rend = hd.Sa = hd.La = hd.off = 0;
        hd.Rn = hd.Sn = hd.Ln = hd.slots = 0;
        hd.fb = hd.nfb = hd.nfa = 0;
        hd.n_in = hd.n_new = hd.nc = 0;
        hd.cls = kClsSkip;
        hd.b = -1;
        hd.i = 0;
        hd.C = 0;
        hd.dtdx_f = 0.0f;
        hd.edges = 0;
        const int b = E.cell_inst[g];
        if (b >= 0) {
            const InstDev &I = E.inst[b];
            const int i = g - I.cell_base - 1;
            const uint32_t step_next = I.step + (update ? 1u : 0u);
            hd.b = b;
            hd.i = i;
            hd.C = I.C;
            hd.dtdx_f = I.dtdx_f;
            hd.edges = (I.bc_left == kBcPhantom ? 1 : 0) | (I.bc_right == kBcPhantom ? 2 : 0);
            if (i < 0 || i >= I.C) {
                const int side = (i < 0) ? 0 : 1;
                const int bc = side ? I.bc_right : I.bc_left;
                if (bc == 0) {
                    double qg[5];
                    const bool ok = ghost_prim(I, side, qg, false, qg);
                    const double Pg = split_fraction(I, qg, ok);
                    myslots = ok ? resample_count(I, cell_id(I, i), step_next, Pg, qg[0]) : 0;
                    for (int k = 0; k < 5; ++k) E.prim[5 * g + k] = qg[k];
                    E.valid[g] = ok ? 1 : 0;
                    E.P[g] = Pg;
                    hd.cls = kClsReservoir;
                    hd.n_new = static_cast<int32_t>(myslots);
                }
                E.cnt[g] = 0;
            } else {
                // particles arriving in g and the sums of what they carry
                int farn = 0, lo = 0, mid = 0;
                double fsum[4] = {0, 0, 0, 0};
                const int nf = E.far_count[1];
                if (nf > 0) {
                    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
                    lo = far_lower(fs, nf, g, INT32_MIN);
                    mid = far_lower(fs, nf, g, g + 1);
                    const int hi = far_lower(fs, nf, g + 1, INT32_MIN);
                    farn = hi - lo;
                    for (int k = lo; k < hi; ++k) {
                        const double u = fs[k].rec.u, v = fs[k].rec.v, w = fs[k].rec.w;
                        fsum[0] += u; fsum[1] += v; fsum[2] += w; fsum[3] += 0.5 * (u * u + v * v + w * w);
                    }
                    hd.fb = lo;
                    hd.nfb = mid - lo;
                    hd.nfa = hi - mid;
                }
                hd.Rend = E.off[q][g - 1] + 2 * static_cast<int64_t>(E.slotsb[q][g - 1]);
                hd.Rn = E.nR[q][g - 1];
                hd.Sa = E.off[q][g];
                hd.Sn = E.nS[q][g];
                hd.La = E.off[q][g + 1] + E.slotsb[q][g + 1];
                hd.Ln = E.nL[q][g + 1];
                const int arrivals = hd.Rn + hd.Sn + hd.Ln + farn;
                double *psi = E.psi + 5 * g;
                if (update) {
                    const int64_t *aR = E.AR + 4 * (g - 1), *aL = E.AL + 4 * (g + 1), *aS = E.Aself + 5 * g;
                    double dp[5];
                    // the three runs' fixed-point sums added as integers and converted once (unless the
                    // sum would overflow)
                    // (conversions by integer operations; the far movers' sums added only where there
                    // are any, the wave fluxes only where one is nonzero: x + 0 and x - 0 are x)
                    dp[0] = fixed_to_double(static_cast<int64_t>(hd.Rn + hd.Ln + farn) + aS[0], 0);
                    for (int k = 0; k < 4; ++k) {
                        const int fr = (k == 3) ? 32 : 40;
                        long long s1, s2;
                        if (add_no_overflow(aR[k], aL[k], s1) && add_no_overflow(s1, aS[k + 1], s2)) {
                            dp[k + 1] = fixed_to_double(s2, fr);
                            if (farn > 0) dp[k + 1] = dp[k + 1] + fsum[k];
                        } else {
                            dp[k + 1] = fixed_to_double(aR[k], fr) + fixed_to_double(aL[k], fr) + fsum[k] +
                                        fixed_to_double(aS[k + 1], fr);
                        }
                    }
                    const double *Fl = E.flux + 5 * (g - 1), *Fr = E.flux + 5 * g;
                    bool zero_flux = true;
                    for (int k = 0; k < 5; ++k) zero_flux = zero_flux && dbl_is_zero(Fl[k]) && dbl_is_zero(Fr[k]);
                    for (int k = 0; k < 5; ++k) {
                        const double fp = I.mp_over_dx * dp[k];
                        if (zero_flux) {
                            psi[k] = psi[k] + fp;
                        } else {
                            const double fw = I.dtdx * (Fr[k] - Fl[k]);
                            psi[k] = psi[k] + fp - fw;
                        }
                    }
                    if (static_cast<int64_t>(step_next) > static_cast<int64_t>(I.avg_start)) {
                        for (int k = 0; k < 5; ++k) E.avg[5 * g + k] += psi[k];
                    }
                }
                double qq[5];
                const bool ok = prim_from_cons(psi, I.inv_cv, qq);
                for (int k = 0; k < 5; ++k) E.prim[5 * g + k] = qq[k];
                E.valid[g] = ok ? 1 : 0;
                const double P = split_fraction(I, qq, ok);
                E.P[g] = P;
                int64_t extra = 0;
                if (ok) {
                    if (dbl_is_zero(P)) {
                        extra = resample_count(I, cell_id(I, i), step_next, 0.0,
                                               psi[0] - fixed_to_double(arrivals, 0) * I.mp_over_dx);
                    } else {
                        extra = static_cast<int64_t>(floor(((1.0 - P) * fmax(psi[0], 0.0)) * I.dx_over_mp)) + 2;
                    }
                }
                E.cnt[g] = arrivals;
                myslots = arrivals + extra;
                hd.n_in = arrivals;
                if (dbl_gt(P, 0.0)) {
                    hd.cls = kClsStaged;
                } else {
                    const int64_t n_tot = arrivals + extra;
                    const int64_t nc = ntc_candidates(I, cell_id(I, i), step_next,
                                                      static_cast<int>(n_tot), psi[0], E.cmax[g], E.fmaj[g]);
                    hd.n_new = static_cast<int32_t>(extra);
                    if (nc < 0 || n_tot > INT32_MAX) {
                        set_err(E.err, kErrOverflow);
                        hd.cls = kClsSkip;
                    } else {
                        hd.nc = static_cast<int32_t>(nc);
                        hd.cls = (nc == 0) ? kClsStream : kClsDirect;
                    }
                }
            }
        }
        if (myslots > INT32_MAX / 2) {
            set_err(E.err, kErrOverflow);
            myslots = 0;
            hd.cls = kClsSkip;
        }
        hd.slots = static_cast<int32_t>(myslots);
        E.slots[g] = static_cast<int32_t>(myslots);
        E.hdr[g] = hd;
    }
    // block sum of the slot bounds
    int64_t x = myslots;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < B / 32; ++w) s += s_w[w];
        E.blocksum[blockIdx.x] = 2 * s;
    }
}

// ------------------------------------------------------------------------------------------
// Offsets of the next step's output blocks, the collision kernel's work list, and the wave flux of
// every interface.  With 256-cell blocks (large pools) at 64 registers (a full SM of warps): the
// double-precision flux, which spills there, runs only where P_f > 0, and the offsets and lists
// before it are latency-bound.  Smaller blocks (small pools, one or two blocks per SM) take up to
// 128 registers and keep the flux's double-precision chain out of local memory.
// ------------------------------------------------------------------------------------------
// Whether a cell's collisions are long dependency chains, which the block kernel runs in parallel
// rounds: at least kHeavyCandidates NTC candidates (Appendix A) on a list that fits the block's
// shared-memory table.  (On longer lists the pairs rarely share a particle and the collision kernel's
// warp takes them 32 at a time.)  A staged cell is estimated with about (1 - P) of its mass in
// particles after absorption and re-sampling.  Only the choice of kernel depends on this, never a
// result.
__device__ __forceinline__ bool staged_is_heavy(const EngineDev &E, int g)
{
    const InstDev &I = E.inst[E.hdr[g].b];
    const double rho_t = E.psi[5 * g];
    const double n_est = (1.0 - E.P[g]) * fmax(rho_t, 0.0) * I.dx_over_mp;
    if (!(n_est <= 0.9 * kBlockSlots)) return false;
    const double rr = (I.ntc_rate == 1) ? rho_t * I.inv_rho_ref : n_est * I.ntc_rr;
    const double nsel = I.ntc_A * rr * (n_est - 1.0) * E.fmaj[g] * E.cmax[g];
    return nsel >= static_cast<double>(kHeavyCandidates);
}

// Chunks of cell g appended to a sample list (lanes of a warp together: one atomic per warp).
__device__ __forceinline__ void append_chunks(const EngineDev &E, int2 *list, int len_ticket, int g, int chunks, int lane)
{
    int incl = chunks;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total > 0) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&E.ticket[len_ticket], total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const int first = base + incl - chunks;
        for (int c = 0; c < chunks; ++c) {
            if (first + c < E.wls_cap) list[first + c] = make_int2(g, c * kSampleChunk);
            else set_err(E.err, kErrOverflow);
        }
    }
}

// Wave flux of the interface after cell g (between local cells i and i+1; -1: the left end), and
// the instance's step counter advanced once per step.
__device__ __forceinline__ void interface_flux(const EngineDev &E, int g)
{
    if (g >= E.G_run) return;
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
        } else if (I.bc_left == kBcPhantom) {
            // the neighbouring part's edge cell, copied into the phantom cell g
            for (int k = 0; k < 5; ++k) a[k] = E.prim[5 * g + k];
            aok = E.valid[g] != 0;
        } else {
            aok = ghost_prim(I, 0, c, cok, a);
        }
    }
    if (gr < 0) {
        if (periodic) {
            const int gg = I.cell_base + 1;
            for (int k = 0; k < 5; ++k) c[k] = E.prim[5 * gg + k];
            cok = E.valid[gg] != 0;
        } else if (I.bc_right == kBcPhantom) {
            for (int k = 0; k < 5; ++k) c[k] = E.prim[5 * (g + 1) + k];
            cok = E.valid[g + 1] != 0;
        } else {
            cok = ghost_prim(I, 1, a, aok, c);
        }
    }
    if (I.recon_mode == 1) {
        // the states beyond a and c, as the flux sees them, and whether a and c have slopes
        const bool use0 = periodic || i >= 0, use1 = periodic || i + 1 < I.C;
        const int g0 = I.cell_base + 1;            // local cell 0
        double wm[5] = {0, 0, 0, 0, 0}, w2[5] = {0, 0, 0, 0, 0};
        bool okm = false, ok2 = false;
        if (use0) {
            const int j = i - 1;
            if (j >= 0 || periodic) {
                const int gj = g0 + ((j + I.C) % I.C);
                for (int k = 0; k < 5; ++k) wm[k] = E.prim[5 * gj + k];
                okm = E.valid[gj] != 0;
            } else {
                okm = ghost_prim(I, 0, E.prim + 5 * g0, E.valid[g0] != 0, wm);
            }
        }
        if (use1) {
            const int j = i + 2;
            if (j < I.C || periodic) {
                const int gj = g0 + (j % I.C);
                for (int k = 0; k < 5; ++k) w2[k] = E.prim[5 * gj + k];
                ok2 = E.valid[gj] != 0;
            } else {
                const int gl2 = g0 + I.C - 1;
                ok2 = ghost_prim(I, 1, E.prim + 5 * gl2, E.valid[gl2] != 0, w2);
            }
        }
        double aR[5], cR[5];
        recon_pair(wm, okm, a, aok, c, cok, w2, ok2, use0, use1, aR, cR);
        wave_flux(I, aR, aok, cR, cok, E.flux + 5 * g, a, c);
    } else {
        wave_flux(I, a, aok, c, cok, E.flux + 5 * g, a, c);
    }
}

// End of a step: the instance's step counter (and the count of averaged states) advance, once per
// instance (by the thread of its left reservoir cell).
__device__ __forceinline__ void step_advance(const EngineDev &E, int g)
{
    if (g >= E.G_run) return;
    const int b = E.cell_inst[g];
    if (b < 0) return;
    InstDev &I = E.inst[b];
    if (g - I.cell_base - 1 != -1) return;
    const uint32_t nxt = I.step + 1u;
    if (static_cast<int64_t>(nxt) > static_cast<int64_t>(I.avg_start)) I.navg += 1;
    I.step = nxt;
}

template <int B>
__global__ void __launch_bounds__(B, (B < 256) ? 512 / B : 1024 / B) k_offsets(EngineDev E, int wp, int advance,
                                                                                 int per)
{
    wait_predecessor();
    __shared__ int64_t s_w[B / 32];
    __shared__ int64_t s_pre;
    const int g = blockIdx.x * B + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // sum of the slot bounds of all earlier blocks (the cell kernel's block sums, `per` of its
    // blocks to one of these)
    int64_t acc = 0;
    for (int j = threadIdx.x; j < blockIdx.x * per; j += B) acc += E.blocksum[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) s_w[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < B / 32; ++w) s += s_w[w];
        s_pre = s;
    }
    __syncthreads();
    // exclusive scan of the slots inside the block
    const int64_t v = (g < E.G_run) ? 2 * static_cast<int64_t>(E.slots[g]) : 0;
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
    bool listed = false;
    int lq = kWarpList;   // work list (kLightList: direct cells with up to kMaxDirect candidates and
                          // nothing re-sampled; kHeavyList: the cells with many candidates)
    int chunks = 0, pchunks = 0;
    if (g < E.G_run) {
        const int64_t o = s_pre + wpre + x - v;
        E.off[wp][g] = o;
        E.hdr[g].off = o;
        if (o + v > E.capacity) {
            set_err(E.err, kErrOverflow);
            E.hdr[g].cls = kClsSkip;
        } else {
            const int cls = E.hdr[g].cls;
            listed = (cls == kClsDirect) || (cls == kClsStaged);
            if (cls == kClsStaged && staged_is_heavy(E, g)) lq = kHeavyList;
            if (cls == kClsDirect) {
                const int nc = E.hdr[g].nc;
                if (nc >= kHeavyCandidates) lq = kHeavyList;
                else if (light_resampling(E.hdr[g]) && nc <= kMaxDirect) lq = kLightList;
            }
            const bool many = E.hdr[g].n_new >= kPreSampleMin;
            // the few re-sampled particles of cells without collisions, and every reservoir's, are
            // drawn in the collision kernel's tail (beside the collisions)
            if (cls == kClsReservoir || (cls == kClsStream && !many))
                chunks = (E.hdr[g].n_new + kSampleChunk - 1) / kSampleChunk;
            if ((cls == kClsDirect || cls == kClsStream) && many && lq != kHeavyList) {
                // many particles to draw (all of them in a first step): drawn ahead over the whole
                // GPU instead of by the one warp that collides the cell.  (The block kernel's cells
                // draw their own: that kernel then depends on nothing of the sampling kernel and
                // starts beside it.)
                pchunks = (E.hdr[g].n_new + kSampleChunk - 1) / kSampleChunk;
                if (cls == kClsDirect) E.hdr[g].edges |= kEdgePresampled;
            }
        }
    }
    // sample lists (one atomic per warp): chunk c of cell g starts at particle c * kSampleChunk
    append_chunks(E, E.wls, kSampleLen, g, chunks, lane);
    append_chunks(E, E.wlp, kPreLen, g, pchunks, lane);
    // work lists of the collision kernels (one atomic per warp and list)
    int light_base = 0;
#pragma unroll
    for (int q = 0; q < kLists; ++q) {
        const bool mine = listed && lq == q;
        const unsigned lm = __ballot_sync(0xffffffffu, mine);
        if (lm) {
            int base = 0;
            if (lane == __ffs(lm) - 1) base = atomicAdd(&E.ticket[kListLen + q], __popc(lm));
            base = __shfl_sync(0xffffffffu, base, __ffs(lm) - 1);
            const int pos = base + __popc(lm & ((1u << lane) - 1u));
            if (mine) E.wl[static_cast<size_t>(q) * E.G + pos] = g;
            if (q == kLightList) {
                light_base = base;
                if (mine) E.wlnc[pos] = E.hdr[g].nc;
            }
        }
    }
    if (g == 0) {
        for (int q = 0; q < kLists; ++q) E.ticket[q] = 0;
        E.ticket[kSampleCtr] = 0;
        E.ticket[kPreCtr] = 0;
        E.ticket[kRoundCtr] = 0;
    }
    if (advance) step_advance(E, g);
    // this warp's light cells (consecutive in the light list), packed into rounds by k_sample
    {
        const unsigned lm = __ballot_sync(0xffffffffu, listed && lq == kLightList);
        if (lane == 0 && g < E.G) E.wgrp[g >> 5] = make_int2(lm ? light_base : 0, __popc(lm));
    }
}

// Wave flux at every interface (Sec. 3.3) from the primitive states of the cell kernel: run at the
// start of the step that applies it (by the cell kernel), on a side stream beside that step's
// collision and streaming kernels, which neither read the flux nor write the states it reads.
template <int B>
__global__ void __launch_bounds__(B, (B < 256) ? 512 / B : 1024 / B) k_flux(EngineDev E)
{
    wait_predecessor();
    interface_flux(E, blockIdx.x * B + threadIdx.x);
}

// ------------------------------------------------------------------------------------------
// Initial cells of one instance: all wave (Psi_p = 0), Psi_t from the two-state profile.
// ------------------------------------------------------------------------------------------
// Initial state of cell g = g0 + t of instance b (all wave, no particles; the left or right state by
// the cell centre's side of x_split).
__device__ __forceinline__ void init_cell(const EngineDev &E, int b, int g, const double *lc, const double *rc,
                                          double x_min, double x_split)
{
    const InstDev &I = E.inst[b];
    E.cell_inst[g] = b;
    const int i = g - I.cell_base - 1;
    for (int p = 0; p < 2; ++p) { E.nL[p][g] = 0; E.nS[p][g] = 0; E.nR[p][g] = 0; E.off[p][g] = 0; E.slotsb[p][g] = 0; }
    for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0; E.AR[4 * g + k] = 0; }
    for (int k = 0; k < 5; ++k) { E.Aself[5 * g + k] = 0; E.avg[5 * g + k] = 0.0; E.flux[5 * g + k] = 0.0; E.psi[5 * g + k] = 0.0; E.prim[5 * g + k] = 0.0; }
    E.ncand[g] = 0; E.nacc[g] = 0; E.nabs[g] = 0; E.nnew[g] = 0; E.cnt[g] = 0; E.slots[g] = 0; E.valid[g] = 0; E.P[g] = 0.0; E.cmax[g] = 0.0; E.fmaj[g] = 1.0;
    if (i < 0 || i >= I.C) return;
    const double xc = x_min + (static_cast<double>(I.id0 + i) + 0.5) * I.dx;
    const bool left = xc < x_split;
    for (int k = 0; k < 5; ++k) E.psi[5 * g + k] = left ? lc[k] : rc[k];
    const double T = left ? I.left[4] : I.right[4];
    E.cmax[g] = 5.0 * sqrt(2.0 * I.R * T);
    E.fmaj[g] = majorant_factor(I, E.cmax[g]);
}

__global__ void k_init_cells(EngineDev E, int b, int g0, int n, double l0, double l1, double l2, double l3, double l4,
                             double r0, double r1, double r2, double r3, double r4, double x_min, double x_split)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double lc[5] = {l0, l1, l2, l3, l4}, rc[5] = {r0, r1, r2, r3, r4};
    init_cell(E, b, g0 + t, lc, rc, x_min, x_split);
}

struct InitCellsBatch {
    InitCellsItem it[kInitBatch];
};

// blockIdx.y: the item (instance); blockIdx.x: cells of that instance
__global__ void k_init_cells_batch(EngineDev E, const __grid_constant__ InitCellsBatch B, int n_items)
{
    const int j = blockIdx.y;
    if (j >= n_items) return;
    const InitCellsItem &q = B.it[j];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= q.n) return;
    init_cell(E, q.b, q.g0 + t, q.lc, q.rc, q.x_min, q.x_split);
}

// ------------------------------------------------------------------------------------------
// Gather of the stable sorted list of instance b (inspection).
// ------------------------------------------------------------------------------------------
template <typename Rec>
__global__ void k_gather(EngineDev E, int rp, int g0, int ncell, const int64_t *start, int64_t total, const int64_t *gate,
                         int32_t *cell, double *xl, double *u, double *v, double *w)
{
    const int t = blockIdx.x;
    if (t >= ncell) return;
    if (gate && *gate != total) return;     // the count differs from the caller's size: write nothing
    const int g = g0 + t;
    const Rec *in = static_cast<const Rec *>(E.buf[rp]);
    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
    const int nf = E.far_count[1];
    int lo = 0, mid = 0, hi = 0;
    if (nf > 0) {
        lo = far_lower(fs, nf, g, INT32_MIN);
        mid = far_lower(fs, nf, g, g + 1);
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
// Normal stress Pi = S_xx and heat flux Q = Q_x of interior cells (Eq. gkt_moment1; inspection,
// not part of the step): the particle part from the central moments of the arrived particles about
// the total velocity U_t,
//   S_p = (m_p/dx) sum (xi_x - U)^2 - rho_p R T_t,   Q_p = (m_p/dx) sum (xi_x - U) |xi - U|^2 / 2,
// rho_p = n m_p / dx; the wave part its NS stress and heat flux (the values of the Chapman-Enskog
// re-sampling: neighbour states as the wave flux sees them, mu_e = eps mu) weighted by
// rho_w / rho_t.  A cell whose total state is not usable reports 0.
// Three passes: one thread per cell splits -U into float pairs; one warp per cell sums its particles
// (single-precision records in double-single arithmetic: the double-precision units are a small
// fraction of the single-precision ones); one thread per cell finishes in double precision.
// ------------------------------------------------------------------------------------------
struct ShCell {
    float nu[6];      // -U, -V, -W as double-single pairs
    double s[2];      // sum (xi_x - U)^2, sum (xi_x - U) |xi - U|^2 / 2 (as (hi, lo) floats for FP32 records)
};

__device__ __forceinline__ bool sh_interior(const EngineDev &E, int g, int &b, int &i)
{
    b = E.cell_inst[g];
    if (b < 0) return false;
    i = g - E.inst[b].cell_base - 1;
    return i >= 0 && i < E.inst[b].C;
}

__global__ void k_sh_split(EngineDev E, int g0, int ncell, ShCell *tmp)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    const int g = g0 + t;
    int b, i;
    if (!sh_interior(E, g, b, i) || !E.valid[g]) return;
    for (int d = 0; d < 3; ++d) {
        const ds x = ds_neg(ds_of_double(E.prim[5 * static_cast<int64_t>(g) + 1 + d]));
        tmp[g].nu[2 * d] = x.hi;
        tmp[g].nu[2 * d + 1] = x.lo;
    }
}

template <typename Rec>
__global__ void k_sh_sums(EngineDev E, int rp, int g0, int ncell, ShCell *tmp)
{
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= ncell) return;
    const int g = g0 + t;
    int b, i;
    if (!sh_interior(E, g, b, i) || !E.valid[g]) return;
    Rec *in = static_cast<Rec *>(E.buf[rp]);
    FarItem<Rec> *fs = static_cast<FarItem<Rec> *>(E.far_sorted);
    const CellHdr h = E.hdr[g];
    const int n = h.n_in;
    constexpr int kIn = 4;   // records per lane in flight
    if constexpr (sizeof(Rec().u) == 4) {
        // single-precision records: c = xi - U formed exactly (TwoSum with the double-single -U) and
        // rounded once, the two terms in single precision, each lane's sums compensated (TwoSum of
        // every addition, the errors summed apart); the arrived runs read as contiguous ranges
        const float v0h = tmp[g].nu[0], v0l = tmp[g].nu[1], v1h = tmp[g].nu[2], v1l = tmp[g].nu[3],
                    v2h = tmp[g].nu[4], v2l = tmp[g].nu[5];
        float s2 = 0.0f, e2 = 0.0f, s3 = 0.0f, e3 = 0.0f;
        auto add = [&](const Rec &r) {
            const ds ax = ds_two_sum(r.u, v0h), ay = ds_two_sum(r.v, v1h), az = ds_two_sum(r.w, v2h);
            const float cx = ax.hi + (ax.lo + v0l), cy = ay.hi + (ay.lo + v1l), cz = az.hi + (az.lo + v2l);
            const float xx = cx * cx;
            const float c2 = fmaf(cz, cz, fmaf(cy, cy, xx));
            const float t3 = (0.5f * cx) * c2;
            const ds a2 = ds_two_sum(s2, xx), a3 = ds_two_sum(s3, t3);
            s2 = a2.hi;
            e2 += a2.lo;
            s3 = a3.hi;
            e3 += a3.lo;
        };
        auto range = [&](const Rec *p, int cnt) {
            for (int k0 = lane; k0 < cnt; k0 += 32 * kIn) {
                Rec x[kIn];
#pragma unroll
                for (int u = 0; u < kIn; ++u)
                    if (k0 + 32 * u < cnt) x[u] = ld_rec(p + k0 + 32 * u);
#pragma unroll
                for (int u = 0; u < kIn; ++u)
                    if (k0 + 32 * u < cnt) add(x[u]);
            }
        };
        range(in + (h.Rend - h.Rn), h.Rn);
        range(in + h.Sa, h.Sn);
        range(in + h.La, h.Ln);
        for (int k = lane; k < h.nfb + h.nfa; k += 32) add(fs[h.fb + k].rec);
        ds f2 = ds_two_sum(s2, e2), f3 = ds_two_sum(s3, e3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f2 = ds_add(f2, {__shfl_xor_sync(0xffffffffu, f2.hi, o), __shfl_xor_sync(0xffffffffu, f2.lo, o)});
            f3 = ds_add(f3, {__shfl_xor_sync(0xffffffffu, f3.hi, o), __shfl_xor_sync(0xffffffffu, f3.lo, o)});
        }
        if (lane == 0) {
            float *o = reinterpret_cast<float *>(tmp[g].s);
            o[0] = f2.hi; o[1] = f2.lo; o[2] = f3.hi; o[3] = f3.lo;
        }
    } else {
        const double *W0 = E.prim + 5 * static_cast<int64_t>(g);
        const double U = W0[1], V = W0[2], Wz = W0[3];
        double s2 = 0.0, s3 = 0.0;
        for (int k0 = lane; k0 < n; k0 += 32 * kIn) {
            Rec x[kIn];
#pragma unroll
            for (int u = 0; u < kIn; ++u) {
                const int r = k0 + 32 * u;
                if (r >= n) break;
                x[u] = ld_rec(arrived_ptr<Rec>(r, h, in, fs));
            }
#pragma unroll
            for (int u = 0; u < kIn; ++u) {
                if (k0 + 32 * u >= n) break;
                const double cx = x[u].u - U, cy = x[u].v - V, cz = x[u].w - Wz;
                s2 += cx * cx;
                s3 += cx * (0.5 * (cx * cx + cy * cy + cz * cz));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        }
        if (lane == 0) { tmp[g].s[0] = s2; tmp[g].s[1] = s3; }
    }
}

__global__ void k_sh_finish(EngineDev E, int fp32, int g0, int ncell, const ShCell *tmp, int accumulate, double *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    const int g = g0 + t;
    int b, i;
    if (!sh_interior(E, g, b, i)) return;
    double pi = 0.0, q = 0.0;
    if (E.valid[g]) {
        const InstDev &I = E.inst[b];
        double s2, s3;
        if (fp32) {
            const float *o = reinterpret_cast<const float *>(tmp[g].s);
            s2 = static_cast<double>(o[0]) + static_cast<double>(o[1]);
            s3 = static_cast<double>(o[2]) + static_cast<double>(o[3]);
        } else {
            s2 = tmp[g].s[0];
            s3 = tmp[g].s[1];
        }
        const double rho_p = static_cast<double>(E.hdr[g].n_in) * I.mp_over_dx;
        pi = I.mp_over_dx * s2 - rho_p * I.R * E.prim[5 * static_cast<int64_t>(g) + 4];
        q = I.mp_over_dx * s3;
        CeCell m;
        ce_coefs(I, E.prim, E.valid, g, i, m);   // sets the stress and heat flux of a usable cell
        const double rho_t = E.psi[5 * static_cast<int64_t>(g)];
        const double wgt = (rho_t - rho_p) / rho_t;
        pi += wgt * m.sxx;
        q += wgt * m.qx;
    }
    if (accumulate) {
        out[g] += pi;
        out[E.G + g] += q;
    } else {
        out[g] = pi;
        out[E.G + g] = q;
    }
}

// ------------------------------------------------------------------------------------------
// Macroscopic profiles of all instances in one pass (inspection): out = [rho | u | T | wave
// fraction] x total, instance b's interior cell i at base[b] + i (base[b] < 0: not reported).
// ------------------------------------------------------------------------------------------
__global__ void k_moments(EngineDev E, int which, const int64_t *base, int64_t total, double *out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= E.G) return;
    const int b = E.cell_inst[g];
    if (b < 0 || base[b] < 0) return;
    const InstDev &I = E.inst[b];
    const int i = g - I.cell_base - 1;
    if (i < 0 || i >= I.C) return;
    const int64_t o = base[b] + i;
    if (o >= total) return;
    const double *c = (which == 1 ? E.avg : E.psi) + 5 * static_cast<int64_t>(g);
    const int64_t navg = I.navg;
    const double scale = (which == 1) ? (navg > 0 ? 1.0 / static_cast<double>(navg) : 0.0) : 1.0;
    // one reciprocal per density instead of five divisions (each double-precision instruction holds
    // an SM sub-partition for 64 cycles on this GPU); the read-out, not a decision of the method
    const double r = c[0] * scale;
    const double mx = c[1] * scale, my = c[2] * scale, mz = c[3] * scale, e5 = c[4] * scale;
    const double ir = r > 0 ? 1.0 / r : 0.0;
    const double ux = mx * ir, uy = my * ir, uz = mz * ir;
    const double tt = r > 0 ? (e5 * ir - 0.5 * (ux * ux + uy * uy + uz * uz)) * I.inv_cv : 0.0;
    const double rt = E.psi[5 * static_cast<int64_t>(g)];
    const double irt = (which == 1) ? (rt > 0 ? 1.0 / rt : 0.0) : ir;
    out[o] = r;
    out[total + o] = ux;
    out[2 * total + o] = tt;
    out[3 * total + o] = rt > 0 ? 1.0 - (static_cast<double>(E.cnt[g]) * I.mp_over_dx) * irt : 0.0;
}

// ------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------
size_t stream_smem_bytes(int fp32, int threads, int groups)
{
    const size_t ring = (groups == 3) ? (fp32 ? sizeof(StreamRing<RecF, 3>) : sizeof(StreamRing<RecD, 3>))
                                      : (fp32 ? sizeof(StreamRing<RecF, 2>) : sizeof(StreamRing<RecD, 2>));
    return static_cast<size_t>(threads / 32) * ((fp32 ? sizeof(StreamShared<RecF>) : sizeof(StreamShared<RecD>)) + ring);
}
size_t stress_tmp_bytes() { return sizeof(ShCell); }
size_t collide_smem_bytes(int fp32)
{
    return (fp32 ? sizeof(CollideShared<RecF>) : sizeof(CollideShared<RecD>)) * (kCollideThreads / 32);
}
int collide_threads() { return kCollideThreads; }

// Sets the kernel's dynamic shared-memory limit to smem_max (the largest any launch shape uses, so
// that engines with different shapes can coexist) and returns blocks per SM at `threads`, `smem`.
template <typename K>
static int occupancy_of(K kern, int threads, size_t smem, size_t smem_max)
{
    int n = 0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_max));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// The streaming kernel for a register budget (variant 0/1/2: 1/2/3 blocks of 512 threads per SM) and
// 2 or 3 record groups per lane.
template <typename Rec>
static void (*stream_kernel(int variant, int groups))(EngineDev, int)
{
    if (groups == 3) {
        if (variant == 2) return k_stream<Rec, 3, 3>;
        if (variant == 1) return k_stream<Rec, 2, 3>;
        return k_stream<Rec, 1, 3>;
    }
    if (variant == 2) return k_stream<Rec, 3, 2>;
    if (variant == 1) return k_stream<Rec, 2, 2>;
    return k_stream<Rec, 1, 2>;
}

int stream_occupancy(int fp32, int variant, int groups, int threads)
{
    // the limit: the largest shape's shared memory, within what a block may opt in to
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const size_t smem = stream_smem_bytes(fp32, threads, groups);
    if (smem > static_cast<size_t>(optin)) return 0;
    const size_t mx = std::min(stream_smem_bytes(fp32, 512, 3), static_cast<size_t>(optin));
    return fp32 ? occupancy_of(stream_kernel<RecF>(variant, groups), threads, smem, mx)
                : occupancy_of(stream_kernel<RecD>(variant, groups), threads, smem, mx);
}

size_t staged_smem_bytes(int fp32)
{
    return fp32 ? sizeof(BlockShared<RecF>) : sizeof(BlockShared<RecD>);
}

// The block kernel at five blocks per SM (96 registers) or, wide, four (128 registers, fewer spills).
int staged_occupancy(int fp32, int wide)
{
    const size_t smem = staged_smem_bytes(fp32);
    if (wide)
        return fp32 ? occupancy_of(k_cellblock<RecF, 4>, kBlockThreads, smem, smem)
                    : occupancy_of(k_cellblock<RecD, 4>, kBlockThreads, smem, smem);
    return fp32 ? occupancy_of(k_cellblock<RecF, 5>, kBlockThreads, smem, smem)
                : occupancy_of(k_cellblock<RecD, 5>, kBlockThreads, smem, smem);
}

int sample_occupancy(int fp32)
{
    return fp32 ? occupancy_of(k_sample<RecF>, kSampleThreads, 0, 0) : occupancy_of(k_sample<RecD>, kSampleThreads, 0, 0);
}

int collide_occupancy(int fp32)
{
    const size_t smem = collide_smem_bytes(fp32);
    return fp32 ? occupancy_of(k_collide<RecF>, kCollideThreads, smem, smem)
                : occupancy_of(k_collide<RecD>, kCollideThreads, smem, smem);
}

namespace {
// Launch with a scheduling priority (blocks of higher-priority launches are dispatched first) and
// programmatic stream serialization (see wait_predecessor).
template <typename... Args>
cudaError_t launch_prio(void (*kernel)(Args...), int grid, int threads, size_t smem, cudaStream_t s, int prio,
                        Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
}  // namespace


// Launch with programmatic stream serialization (see wait_predecessor).
template <typename... Args>
static cudaError_t launch_pdl(void (*kernel)(Args...), dim3 grid, int threads, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
cudaError_t launch_sample(const EngineDev &E, int fp32, int rp, int grid, cudaStream_t s, int prio)
{
    const cudaError_t e = fp32 ? launch_prio(k_sample<RecF>, grid, kSampleThreads, 0, s, prio, E, rp)
                               : launch_prio(k_sample<RecD>, grid, kSampleThreads, 0, s, prio, E, rp);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_collide(const EngineDev &E, int fp32, int rp, int grid, cudaStream_t s, int prio)
{
    const size_t smem = collide_smem_bytes(fp32);
    cudaError_t e = fp32 ? launch_prio(k_collide<RecF>, grid, kCollideThreads, smem, s, prio, E, rp)
                         : launch_prio(k_collide<RecD>, grid, kCollideThreads, smem, s, prio, E, rp);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_staged(const EngineDev &E, int fp32, int wide, int rp, int grid, cudaStream_t s, int prio)
{
    const size_t smem = staged_smem_bytes(fp32);
    cudaError_t e;
    if (wide)
        e = fp32 ? launch_prio(k_cellblock<RecF, 4>, grid, kBlockThreads, smem, s, prio, E, rp)
                 : launch_prio(k_cellblock<RecD, 4>, grid, kBlockThreads, smem, s, prio, E, rp);
    else
        e = fp32 ? launch_prio(k_cellblock<RecF, 5>, grid, kBlockThreads, smem, s, prio, E, rp)
                 : launch_prio(k_cellblock<RecD, 5>, grid, kBlockThreads, smem, s, prio, E, rp);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_stream(const EngineDev &E, int fp32, int variant, int groups, int rp, int threads, cudaStream_t s,
                          int prio)
{
    const int wpb = threads / 32;
    const int grid = (E.G_run + wpb - 1) / wpb;
    const size_t smem = stream_smem_bytes(fp32, threads, groups);
    const cudaError_t e = fp32 ? launch_prio(stream_kernel<RecF>(variant, groups), grid, threads, smem, s, prio, E, rp)
                               : launch_prio(stream_kernel<RecD>(variant, groups), grid, threads, smem, s, prio, E, rp);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_far_sort(const EngineDev &E, int fp32, cudaStream_t s)
{
    const int grid = (E.far_cap + 255) / 256;
    if (fp32) launch_pdl(k_far_sort<RecF>, dim3(grid), 256, s, E);
    else launch_pdl(k_far_sort<RecD>, dim3(grid), 256, s, E);
    return cudaGetLastError();
}

// Cells per block of the offset and flux kernels (and of the cell kernel on small pools).  Their
// per-cell work is a chain of double-precision operations (primitive state, Eq. (p), the wave flux),
// and an SM's double-precision units are few: a small pool is spread over as many SMs as it can fill
// (two blocks each) instead of a few full blocks.
static int cell_block(int cells, int nsm)
{
    for (int b = kCellBlockMin; b < kCellBlock; b *= 2)
        if (cells <= b * 2 * nsm) return b;
    return kCellBlock;
}

// Cells per block of the cell kernel alone: on a large pool, blocks of kCellBlockLarge instead of
// kCellBlock spread its double-precision chains evenly over the SMs' sub-partitions (all blocks are
// resident at once; with 256-cell blocks some SMs hold a block more than others).  The offset
// kernel keeps its own blocks and reads the cell kernel's block sums in their units.
static int cells_kernel_block(int cells, int nsm)
{
    const int b = cell_block(cells, nsm);
    return b == kCellBlock ? kCellBlockLarge : b;
}

template <typename Rec>
static cudaError_t launch_cells_b(const EngineDev &E, int b, int grid, int q, int update, cudaStream_t s)
{
    if (b == 32) launch_pdl(k_cells<Rec, 32>, dim3(grid), 32, s, E, q, update);
    else if (b == 64) launch_pdl(k_cells<Rec, 64>, dim3(grid), 64, s, E, q, update);
    else if (b == 128) launch_pdl(k_cells<Rec, 128>, dim3(grid), 128, s, E, q, update);
    else launch_pdl(k_cells<Rec, kCellBlock>, dim3(grid), kCellBlock, s, E, q, update);
    return cudaGetLastError();
}

cudaError_t launch_cells(const EngineDev &E, int fp32, int q, int update, cudaStream_t s)
{
    const int b = cells_kernel_block(E.G_run, E.nsm > 0 ? E.nsm : 1);
    const int grid = (E.G_run + b - 1) / b;
    return fp32 ? launch_cells_b<RecF>(E, b, grid, q, update, s) : launch_cells_b<RecD>(E, b, grid, q, update, s);
}

cudaError_t launch_offsets(const EngineDev &E, int wp, int advance, cudaStream_t s)
{
    const int nsm = E.nsm > 0 ? E.nsm : 1;
    const int b = cell_block(E.G_run, nsm);
    const int per = b / cells_kernel_block(E.G_run, nsm);
    const int grid = (E.G_run + b - 1) / b;
    if (b == 32) launch_pdl(k_offsets<32>, dim3(grid), 32, s, E, wp, advance, per);
    else if (b == 64) launch_pdl(k_offsets<64>, dim3(grid), 64, s, E, wp, advance, per);
    else if (b == 128) launch_pdl(k_offsets<128>, dim3(grid), 128, s, E, wp, advance, per);
    else launch_pdl(k_offsets<kCellBlock>, dim3(grid), kCellBlock, s, E, wp, advance, per);
    return cudaGetLastError();
}

cudaError_t launch_flux(const EngineDev &E, cudaStream_t s, int prio)
{
    const int b = cell_block(E.G_run, E.nsm > 0 ? E.nsm : 1);
    const int grid = (E.G_run + b - 1) / b;
    cudaError_t e;
    if (b == 32) e = launch_prio(k_flux<32>, grid, 32, 0, s, prio, E);
    else if (b == 64) e = launch_prio(k_flux<64>, grid, 64, 0, s, prio, E);
    else if (b == 128) e = launch_prio(k_flux<128>, grid, 128, 0, s, prio, E);
    else e = launch_prio(k_flux<kCellBlock>, grid, kCellBlock, 0, s, prio, E);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_stress_heat(const EngineDev &E, int fp32, int rp, int g0, int ncell, int accumulate, double *out,
                               void *tmp, cudaStream_t s)
{
    if (ncell <= 0) return cudaSuccess;
    ShCell *t = static_cast<ShCell *>(tmp);
    const int gt = (ncell + 255) / 256;
    if (fp32) k_sh_split<<<gt, 256, 0, s>>>(E, g0, ncell, t);
    const int gw = (ncell + 3) / 4;   // one warp per cell
    if (fp32) k_sh_sums<RecF><<<gw, 128, 0, s>>>(E, rp, g0, ncell, t);
    else k_sh_sums<RecD><<<gw, 128, 0, s>>>(E, rp, g0, ncell, t);
    k_sh_finish<<<gt, 256, 0, s>>>(E, fp32, g0, ncell, t, accumulate, out);
    return cudaGetLastError();
}

cudaError_t launch_init_turn(cudaStream_t s)
{
    k_init_turn<<<1, (kTurnTable > kLogTable ? kTurnTable : kLogTable), 0, s>>>();
    return cudaGetLastError();
}

cudaError_t launch_init_cells_batch(const EngineDev &E, const InitCellsItem *items, int n_items, cudaStream_t s)
{
    for (int j0 = 0; j0 < n_items; j0 += kInitBatch) {
        const int m = std::min(kInitBatch, n_items - j0);
        InitCellsBatch B;
        int max_n = 0;
        for (int j = 0; j < m; ++j) {
            B.it[j] = items[j0 + j];
            max_n = std::max(max_n, items[j0 + j].n);
        }
        if (max_n <= 0) continue;
        const dim3 grid((max_n + 255) / 256, m);
        k_init_cells_batch<<<grid, 256, 0, s>>>(E, B, m);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_init_cells(const EngineDev &E, int b, int g0, int n, const double *lc, const double *rc, double x_min,
                              double x_split, cudaStream_t s)
{
    const int grid = (n + 255) / 256;
    k_init_cells<<<grid, 256, 0, s>>>(E, b, g0, n, lc[0], lc[1], lc[2], lc[3], lc[4], rc[0], rc[1], rc[2], rc[3], rc[4],
                                      x_min, x_split);
    return cudaGetLastError();
}

cudaError_t launch_moments(const EngineDev &E, int which, const int64_t *d_base, int64_t total, double *d_out,
                           cudaStream_t s)
{
    k_moments<<<(E.G + 255) / 256, 256, 0, s>>>(E, which, d_base, total, d_out);
    return cudaGetLastError();
}

cudaError_t launch_gather(const EngineDev &E, int fp32, int rp, int b, int g0, int ncell, const int64_t *d_start,
                          int64_t total, const int64_t *gate, int32_t *cell, double *xl, double *u, double *v,
                          double *w, cudaStream_t s)
{
    (void)b;
    if (ncell <= 0) return cudaSuccess;
    if (fp32) k_gather<RecF><<<ncell, 128, 0, s>>>(E, rp, g0, ncell, d_start, total, gate, cell, xl, u, v, w);
    else k_gather<RecD><<<ncell, 128, 0, s>>>(E, rp, g0, ncell, d_start, total, gate, cell, xl, u, v, w);
    return cudaGetLastError();
}

}  // namespace duwp

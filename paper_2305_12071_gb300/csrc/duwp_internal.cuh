// duwp_internal.cuh -- device data layout and per-particle / per-cell arithmetic of the DUWP step
// (Cao, Liu, Yang, Zhong, arXiv 2305.12071, Sec. 3.4 and Appendix A) for sm_103a.
//
// Layout in HBM (one engine = a pool of G flattened cells shared by all resident instances):
//   instance b owns cells [cell_base, cell_base + C + 2): left reservoir (ghost), cells 0..C-1,
//   right reservoir.  Particles are 16-byte (FP32: xl, u, v, w) or 32-byte (FP64) records in two
//   buffers used alternately.  After a step every cell s owns one output block (twice its slot
//   bound) in the write buffer, holding its particles that stayed (S, forward from the start),
//   moved one cell left (L, forward from the middle) and moved one cell right (R, backward from
//   the end), each run in the order the particles had before transport.  The stable sorted list
//   of a cell g for the next step is then  [far movers from cells < g-1] R(g-1) S(g) L(g+1)
//   [far movers from cells > g+1]  -- exactly the stable counting-sort order by new cell, without
//   a global sort pass.  Particles that moved two or more cells (or wrapped around a periodic
//   domain) go to a small list sorted separately.
//
// Every decision-bearing operation (transport, index picks, acceptance, counts) follows one fixed
// operation order, and the library is compiled with -fmad=false; fused multiply-adds appear only
// where written explicitly.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "duwp_dsmath.cuh"

namespace duwp {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.283185307179586;

// Boundary kind of an instance's end that faces another part of the same domain (a domain split into
// cell ranges): no wall, no reservoir; the cell beyond the end is a phantom of the neighbouring
// part's edge cell, whose state and incoming particle runs are copied in between the kernels.
constexpr int kBcPhantom = 4;

// Destination returned by the transport for a particle that left the domain (removed).
constexpr int64_t kGone = INT64_MIN / 2;

// Device error codes (mirrors of the public status values).
constexpr int kErrOverflow = -7;
constexpr int kErrTimeout = -5;

enum Purpose : uint32_t { kAbsorb = 1, kRound = 2, kSample = 3, kCollide = 4 };

struct alignas(16) RecF { float xl, u, v, w; };
struct alignas(16) RecD { double xl, u, v, w; };

// Per-instance constants and state kept on the device.
struct InstDev {
    int32_t C;              // interior cells
    int32_t cell_base;      // flattened index of the left reservoir cell
    int32_t bc_left, bc_right;
    int32_t eps_mode, flux_mode, ntc_rate, active;
    uint32_t key0, key1;    // generator key (seed)
    int32_t id0;            // global index of local cell 0 (0 unless the instance is one part of a
                            // domain split into cell ranges); generator id of local cell i = id0 + i + 1
    uint32_t step;          // steps completed (advanced once per step, after the cell update)
    int32_t avg_start;
    int64_t navg;           // states accumulated into the time average
    unsigned long long updates;   // particles streamed by this instance (interior cells), all steps
    double dx, dt, dtdx, mp, dx_over_mp, mp_over_dx;
    double R, Pr, omega, T_ref, rho_ref, mu_ref, upsilon, c_ref, ntc_A;
    double ntc_rr;          // m_p / (dx rho_ref): particle density ratio per particle
    double inv_rho_ref;
    double inv_cv;          // 1 / (3/2 R): temperature per unit of specific internal energy
    double vhs_expo;        // 1 - 2 upsilon: exponent of c_r in the VHS acceptance test (Appendix A)
    float vhs_expo_f;
    float dtdx_f;
    // single-precision copies for the estimates (each double-precision instruction, conversions
    // included, holds an SM sub-partition for 64 cycles on this GPU)
    float mu_ref_f, T_ref_f, omega_f, R_f, dt_f;
    int32_t resample_mode;  // 0: Maxwellian re-sampling, 1: with its Chapman-Enskog (NS) correction
    int32_t split_mode;     // 0: Eq. (p), 1: 1 - exp(-dt/tau) (quantified model competition)
    int32_t recon_mode;     // 0: first-order wave states, 1: van Leer limited reconstruction
    double left[5], right[5];   // reservoir primitive states (rho, u, v, w, T)
};

// Sorted list entry of a particle that moved two or more cells (or wrapped): new cell, source
// cell and its position in the source cell's list before transport (the stable-order key).
template <typename Rec>
struct FarItem {
    int32_t dest, src, q, pad;
    Rec rec;
};

// Plan of one cell's particle work in the next step, written by the cell kernels at the end of a
// step (k_cells: lists, counts, class; k_offsets_flux: output block): where the cell's arrived list
// lies in the read buffer, where its output block starts, and the counts that are known before any
// particle is touched (re-sampled count and NTC candidate count when P = 0).
enum CellClass : int32_t {
    kClsSkip = 0,       // unused cell, a reservoir that samples nothing, or a cell in error
    kClsStream = 1,     // P = 0 and no collision candidates: stream the arrived + re-sampled particles
    kClsDirect = 2,     // P = 0 and candidates: re-sample after the arrived positions, collide in
                        // place, stream
    kClsStaged = 3,     // P > 0: absorption, compaction and re-sampling into the output block
    kClsReservoir = 4   // inflow/outflow reservoir: stream the particles sampled at its state
};
constexpr int kMaxDirect = 32;

struct alignas(16) CellHdr {
    int64_t Rend;       // one past the last record of the left neighbour's R run (read backwards)
    int64_t Sa;         // first record of the cell's own S run
    int64_t La;         // first record of the right neighbour's L run
    int64_t off;        // first slot of the cell's output block in the write buffer
    int32_t Rn, Sn, Ln;
    int32_t slots;      // slot bound (the output block holds 2 x slots)
    int32_t fb, nfb, nfa;   // far movers: first sorted index, counts from the left / from the right
    int32_t n_in;       // arrived particles (the list length before absorption)
    int32_t n_new;      // re-sampled particles (classes 1, 2, 4)
    int32_t nc;         // NTC candidates (classes 1, 2)
    int32_t cls;        // CellClass
    int32_t b;          // instance
    int32_t i;          // local cell index (-1 and C: reservoirs)
    int32_t C;          // cells of the instance
    float dtdx_f;       // dt/dx of the instance in single precision (transport of FP32 records)
    int32_t edges;      // bit 0: the left end faces a phantom cell, bit 1: the right end does
};
static_assert(sizeof(CellHdr) == 96, "cell header layout");

// Pointers of one engine, passed by value to every kernel.
struct EngineDev {
    int32_t G;                 // flattened cells in the pool
    int32_t n_inst;
    int64_t capacity;          // particle slots per buffer
    int32_t far_cap;
    int32_t G_run;             // the step kernels cover cells [0, G_run) (<= G): every resident
                               // instance lies below it, the cells above are unused and clean
    int32_t nsm;               // SMs of the device (launch shapes of the cell kernels)
    InstDev *inst;
    int32_t *cell_inst;        // instance of each flattened cell, -1 = unused
    double *psi;               // G x 5 total state Psi_t (reservoirs: unused)
    double *prim;              // G x 5 primitive state (rho, u, v, w, T)
    int32_t *valid;            // G: primitive state usable (rho > 0, T > 0)
    double *P;                 // G: absorption fraction, Eq. (p)
    double *cmax;              // G: NTC majorant
    double *fmaj;              // G: (c_max / c_ref)^{-2 upsilon} of the current c_max
    double *flux;              // G x 5: wave flux at the interface between g and g+1
    double *avg;               // G x 5: time-average accumulator of Psi_t
    // exact fixed-point sums written by the streaming kernel (velocities x 2^40, |xi|^2/2 x 2^32),
    // converted to double by the cell kernel
    int64_t *AL, *AR;          // G x 4: sums (u, v, w, |xi|^2/2) of the L / R runs (post-transport)
    int64_t *Aself;            // G x 5: change of the cell's own particle moments (leavers,
                               // reflections); [0] the count
    int32_t *slots;            // G: upper bound of the cell's list after re-sampling (this step)
    int32_t *slotsb[2];        // G: the bound each output block was written with, per buffer (block = 2 x bound)
    int32_t *cnt;              // G: particles arriving in the cell (list length this step)
    int32_t *nL[2], *nS[2], *nR[2];
    int64_t *off[2];           // G: first slot of each cell's output block, per buffer
    int64_t *blocksum;         // per 256-cell block sums of slots
    int32_t *nnew, *nabs, *ncand, *nacc;
    void *buf[2];
    void *far_app;             // far movers appended during a step (unsorted)
    void *far_sorted;          // the same, sorted by (dest, src, q)
    int32_t *far_count;        // [0]: appended, [1]: sorted
    int32_t *err;              // first device error
    int32_t *ticket;           // collision kernel work counters and list lengths (kTickets, see below)
    CellHdr *hdr;              // G: plan of each cell's particle work in the next step
    int32_t *wl;               // kLists x G: work lists of the collision kernels (the light direct cells,
                               // the other cells of the collision kernel, the heavy cells)
    int2 *wls;                 // sample list: (cell, first index) of chunks of kSampleChunk re-sampled particles
    int2 *wlp;                 // the same for the particles drawn ahead of the collision kernels
    int2 *wgrp;                // G/32: the light cells each warp of k_offsets_flux appended to the light
                               // list (first list position, cells)
    int32_t *wlnc;             // G: NTC candidates of each light-list entry
    int2 *wr;                  // G: rounds of the light list (first list position, cells): consecutive
                               // light cells whose candidates fit in the 32 lanes of a warp
    int32_t wls_cap;           // entries of wls (and of wlp)
};

// ticket[q] (q < kLists): next item of work list q; ticket[kListLen + q]: its length; ticket[kSampleLen]
// and ticket[kSampleCtr]: length of and next item of the sample list.  Lists kLightList and kWarpList
// belong to the collision kernel (the light direct cells, packed several to a warp, and the other
// cells, one warp each), list kHeavyList to the block kernel (the cells with many collision
// candidates, one block per cell).
constexpr int kLists = 3;
constexpr int kLightList = 0;
constexpr int kWarpList = 1;
constexpr int kHeavyList = 2;
constexpr int kListLen = 3;
constexpr int kSampleLen = 6;
constexpr int kSampleCtr = 7;
// ticket[kPreLen] / ticket[kPreCtr]: length of and next item of the list of particles drawn ahead (the
// re-sampled particles of direct cells and of cells without collisions with at least kPreSampleMin of
// them, drawn by k_sample before the collision kernels run; such a direct cell's header carries
// kEdgePresampled in `edges`).  With the threshold at one particle every direct cell that re-samples
// takes the packed light rounds when its candidates allow (the steps after a first step re-sample in
// many cells: 1.078 -> 1.046 ms for the second step of the shock batch, steady steps unchanged).
constexpr int kPreLen = 8;
constexpr int kPreCtr = 9;
constexpr int kPreSampleMin = 1;
// ticket[kRoundLen] / ticket[kRoundCtr]: length of and next item of the round list (wr)
constexpr int kRoundLen = 10;
constexpr int kRoundCtr = 11;
constexpr int kEdgePresampled = 4;
constexpr int kTickets = 16;

// Re-sampled particles of classes 1 and 4 are drawn by the collision kernel in chunks of this many,
// spread over all its warps, and written after the arrived positions of the cell's output block.
constexpr int kSampleChunk = 64;

constexpr int kCellBlock = 256;   // cells per block of the cell / offset kernels (at most)
constexpr int kCellBlockMin = 32; // (at least)
constexpr int kCellBlockLarge = 64;   // cells per block of the cell kernel on a large pool
static_assert(kCellBlock % kCellBlockLarge == 0 && kCellBlockLarge >= kCellBlockMin,
              "the offset kernel reads whole cell-kernel blocks");

// ------------------------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round multiplies words 0
// and 2 by the two round constants (full 64-bit products), swaps the halves across the lanes with
// the key XORed in, and the key is bumped by the Weyl increments after each round.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void philox10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                                         uint32_t c3, uint32_t out[4])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Counter layout: (id, sub, step, purpose); id = local cell index + 1 (reservoirs 0 and C+1).
__device__ __forceinline__ void draw(const InstDev &I, uint32_t id, uint32_t sub, uint32_t step, uint32_t purpose,
                                     uint32_t w[4])
{
    philox10(I.key0, I.key1, id, sub, step, purpose, w);
}

// Generator id of local cell i (-1 and C: the ends) of an instance.
__device__ __forceinline__ uint32_t cell_id(const InstDev &I, int i) { return static_cast<uint32_t>(I.id0 + i + 1); }

// Uniform in [0,1) with 53 random bits: 32 from the first word, 21 from the second.
// (The exact value m 2^-53 is formed by integer operations, without the double-precision unit.)
__device__ __forceinline__ double u53(uint32_t a, uint32_t b)
{
    const uint64_t m = (static_cast<uint64_t>(a) << 21) ^ static_cast<uint64_t>(b >> 11);
    return fixed_to_double(static_cast<int64_t>(m), 53);
}

// Index in [0, n) from a 32-bit word: the high half of the 64-bit product.
__device__ __forceinline__ uint32_t idx32(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// ------------------------------------------------------------------------------------------
// Cell-level quantities (FP64)
// ------------------------------------------------------------------------------------------

// Primitive state from the conservative one (rho, rho U, rho V, rho W, rho E); monatomic gas:
// rho E = rho |U|^2 / 2 + 3/2 rho R T.  Returns whether the state is usable.  One division: the
// quotients are products with 1/rho and 1/(3/2 R), within an ulp of the divisions (the double-precision
// units are few on this GPU, and a division costs about nine of their operations).
__device__ inline bool prim_from_cons(const double *psi, double inv_cv, double *q)
{
    const double rho = psi[0];
    q[0] = rho;
    q[1] = q[2] = q[3] = q[4] = 0.0;
    if (!dbl_gt(rho, 0.0)) return false;
    const double ir = 1.0 / rho;
    const double u = psi[1] * ir, v = psi[2] * ir, w = psi[3] * ir;
    const double e = psi[4] * ir - 0.5 * (u * u + v * v + w * w);
    const double T = e * inv_cv;
    q[1] = u; q[2] = v; q[3] = w; q[4] = T;
    return dbl_gt(T, 0.0) && dbl_finite(T) && dbl_finite(u) && dbl_finite(v) && dbl_finite(w);
}

__device__ inline double viscosity(const InstDev &I, double T) { return I.mu_ref * pow(T / I.T_ref, I.omega); }

// Single-precision estimate of tau = mu(T)/(rho R T); used only where an error far below 1% cannot
// change the decision dt <= tau.  Returns 0 when the estimate is not usable (over/underflow).
__device__ __forceinline__ float tau_estimate(const InstDev &I, float rho, float T)
{
    const float mu = I.mu_ref_f * powf(T / I.T_ref_f, I.omega_f);
    const float tau = mu / (rho * I.R_f * T);
    return (tau > 0.0f && tau < 1e30f) ? tau : 0.0f;
}

// Eq. (p): P = 0 if dt <= tau, else 1 - tau/dt, with tau = mu / p.  When the single-precision
// estimate of tau exceeds dt by more than 1% (its error is below 1e-5 relative), P = 0 without the
// double-precision power.
__device__ inline double split_fraction(const InstDev &I, const double *q, bool ok)
{
    if (!ok) return 0.0;
    if (I.split_mode == 1) {
        // Sec. 3.2: a particle collides during the step with probability 1 - exp(-dt/tau)
        const double tau = viscosity(I, q[4]) / (q[0] * I.R * q[4]);
        return -expm1(-(I.dt / tau));
    }
    const float t32 = tau_estimate(I, f32_of_double(q[0]), f32_of_double(q[4]));
    if (t32 > 1.01f * I.dt_f && dbl_gt(q[0], 1e-30) && dbl_gt(q[4], 1e-30) && dbl_lt(q[4], 1e30)) return 0.0;
    const double tau = viscosity(I, q[4]) / (q[0] * I.R * q[4]);
    if (I.dt <= tau) return 0.0;
    return 1.0 - tau / I.dt;
}

// Number of particles drawn from the wave: stochastic rounding of (1-P) max(rho_w,0) dx / m_p.
__device__ inline int64_t resample_count(const InstDev &I, uint32_t id, uint32_t step, double P, double rho_w)
{
    uint32_t w[4];
    draw(I, id, 0u, step, kRound, w);
    // ((1 - P) max(rho_w, 0)) dx/m_p, with the factor 1 - P = 1 of P = 0 not multiplied (exact)
    const double rw = dbl_gt(rho_w, 0.0) ? rho_w : 0.0;
    const double x = (dbl_is_zero(P) ? rw : (1.0 - P) * rw) * I.dx_over_mp;
    return static_cast<int64_t>(floor(x + u53(w[0], w[1])));
}

// Reservoir (ghost) primitive state beyond the left (side 0) or right (side 1) end.
__device__ inline bool ghost_prim(const InstDev &I, int side, const double *inner, bool inner_ok, double *q)
{
    const int bc = side ? I.bc_right : I.bc_left;
    if (bc == 0) {  // inflow/outflow reservoir at the boundary state
        const double *s = side ? I.right : I.left;
        for (int k = 0; k < 5; ++k) q[k] = s[k];
        return s[0] > 0.0 && s[4] > 0.0;
    }
    if (bc == 1) {  // specular wall: mirror state
        for (int k = 0; k < 5; ++k) q[k] = inner[k];
        q[1] = -inner[1];
        return inner_ok;
    }
    for (int k = 0; k < 5; ++k) q[k] = 0.0;   // vacuum (periodic is handled by the caller)
    return false;
}

// Viscosity correction of the NS flux as a function of x = dt/tau (Sec. 3.3):
// eps1 = 1 - x/(e^x - 1) (Eq. vp1), eps12 = x/(2+x), eps0 = 1, time-averaged eps (Eq. vp).
__device__ inline double eps_factor(int mode, double x)
{
    if (mode == 2) return 1.0;
    if (mode == 1) return x / (2.0 + x);
    if (mode == 3) {
        const double a = -expm1(-x), b = 1.0 + exp(-x);
        return (-2.0 * a + x * b) / (x - a);
    }
    return 1.0 - x / expm1(x);
}

// <u^n> of a unit-density Maxwellian over u > 0 (pos) and u < 0 (neg), n = 0..3, lam = 1/(2RT).
__device__ inline void half_moments(double U, double lam, double *pos, double *neg)
{
    const double s = sqrt(lam);
    pos[0] = 0.5 * erfc(-s * U);
    neg[0] = 0.5 * erfc(s * U);
    const double tail = 0.5 * exp(-lam * U * U) / sqrt(kPi * lam);
    pos[1] = U * pos[0] + tail;
    neg[1] = U * neg[0] - tail;
    const double h = 1.0 / (2.0 * lam);
    pos[2] = U * pos[1] + h * pos[0];
    neg[2] = U * neg[1] + h * neg[0];
    pos[3] = U * pos[2] + 2.0 * h * pos[1];
    neg[3] = U * neg[2] + 2.0 * h * neg[1];
}

// Second-order wave reconstruction (recon_mode 1): per primitive variable the van Leer limited
// slope 2 dl dr / (dl + dr) where the one-sided differences agree in sign, else 0; the interface
// between cells 0 and 1 sees w0 + s0/2 and w1 - s1/2 (use0 / use1 false: that cell has no slope,
// being a reservoir or mirror cell); the cell states are kept if either side would lose rho > 0 or
// T > 0.  Same expressions, in the same order, as the double-precision checker.
__device__ inline void vl_slopes(const double *qa, const double *qb, const double *qc, double *s)
{
    for (int k = 0; k < 5; ++k) {
        const double dl = qb[k] - qa[k], dr = qc[k] - qb[k];
        s[k] = (dl * dr > 0.0) ? (2.0 * dl * dr) / (dl + dr) : 0.0;
    }
}

__device__ inline void recon_pair(const double *wm, bool okm, const double *w0, bool ok0, const double *w1, bool ok1,
                                  const double *w2, bool ok2, bool use0, bool use1, double *L, double *R)
{
    for (int k = 0; k < 5; ++k) { L[k] = w0[k]; R[k] = w1[k]; }
    if (!ok0 || !ok1) return;
    double s0[5] = {0, 0, 0, 0, 0}, s1[5] = {0, 0, 0, 0, 0};
    if (use0 && okm) vl_slopes(wm, w0, w1, s0);
    if (use1 && ok2) vl_slopes(w0, w1, w2, s1);
    double a[5], b[5];
    for (int k = 0; k < 5; ++k) {
        a[k] = w0[k] + 0.5 * s0[k];
        b[k] = w1[k] - 0.5 * s1[k];
    }
    if (a[0] > 0.0 && a[4] > 0.0 && b[0] > 0.0 && b[4] > 0.0)
        for (int k = 0; k < 5; ++k) { L[k] = a[k]; R[k] = b[k]; }
}

// Wave flux through the interface between a left state a and a right state b (per unit area):
// interface equilibrium from the colliding half-Maxwellians, Euler flux of it (or the split
// kinetic flux), NS stress and heat flux with mu_e = eps mu(T0), weighted by
// P_f = max(0, 1 - tau_f/dt) (Sec. 3.3, Eq. ce2 at t = dt; Step 3).
// Single-precision interface state (rho0, T0) of the colliding half-Maxwellians and a bound on
// the cancellation in T0; returns false when the estimate cannot decide P_f = 0.
__device__ inline bool flux_is_zero_estimate(const InstDev &I, const double *a, bool aok, const double *b, bool bok)
{
    float r0 = 0.f, m0 = 0.f, my = 0.f, mz = 0.f, e0 = 0.f;
    const float R = I.R_f;
    for (int side = 0; side < 2; ++side) {
        const double *s = side ? b : a;
        if (!(side ? bok : aok)) continue;
        const float rho = f32_of_double(s[0]), U = f32_of_double(s[1]), V = f32_of_double(s[2]),
                    W = f32_of_double(s[3]), T = f32_of_double(s[4]);
        const float lam = 1.0f / (2.0f * R * T);
        const float sl = sqrtf(lam);
        const float sg = side ? 1.0f : -1.0f;            // left: u > 0 half; right: u < 0 half
        const float M0 = 0.5f * erfcf(sg * sl * U);
        const float tail = -sg * 0.5f * expf(-lam * U * U) / sqrtf(3.14159265f * lam);
        const float M1 = U * M0 + tail;
        const float M2 = U * M1 + M0 / (2.0f * lam);
        r0 += rho * M0;
        m0 += rho * M1;
        my += rho * V * M0;
        mz += rho * W * M0;
        e0 += 0.5f * rho * (M2 + (V * V + W * W + 1.0f / lam) * M0);
    }
    if (!(r0 > 1e-30f)) return false;
    const float U0 = m0 / r0, V0 = my / r0, W0 = mz / r0;
    const float kin = 0.5f * (U0 * U0 + V0 * V0 + W0 * W0);
    const float th = e0 / r0 - kin;
    // cancellation: the relative error of th is about 1e-6 (e0/r0)/th; require it below 1e-3
    if (!(th > 1e-3f * (e0 / r0))) return false;
    const float T0 = th / (1.5f * R);
    const float t32 = tau_estimate(I, r0, T0);
    return t32 > 1.05f * I.dt_f;
}

// ga, gb: the cell states whose difference gives the NS gradients (a, b themselves unless a and b
// are reconstructed interface states).
__device__ inline void wave_flux(const InstDev &I, const double *a, bool aok, const double *b, bool bok,
                                 double *F, const double *ga, const double *gb)
{
    for (int k = 0; k < 5; ++k) F[k] = 0.0;
    // P_f = 0 (no wave flux) is decided in single precision when tau_f exceeds dt by over 5%
    if (I.split_mode == 0 && flux_is_zero_estimate(I, a, aok, b, bok)) return;
    double ap[4] = {0, 0, 0, 0}, an[4] = {0, 0, 0, 0}, bp[4] = {0, 0, 0, 0}, bn[4] = {0, 0, 0, 0};
    double la = 0.0, lb = 0.0, ra = 0.0, rb = 0.0, ta = 0.0, tb = 0.0;
    if (aok) {
        la = 1.0 / (2.0 * I.R * a[4]);
        half_moments(a[1], la, ap, an);
        ra = a[0];
        ta = a[2] * a[2] + a[3] * a[3] + 1.0 / la;
    }
    if (bok) {
        lb = 1.0 / (2.0 * I.R * b[4]);
        half_moments(b[1], lb, bp, bn);
        rb = b[0];
        tb = b[2] * b[2] + b[3] * b[3] + 1.0 / lb;
    }
    const double av = aok ? a[2] : 0.0, aw = aok ? a[3] : 0.0;
    const double bv = bok ? b[2] : 0.0, bw = bok ? b[3] : 0.0;
    const double rho0 = ra * ap[0] + rb * bn[0];
    const double mx0 = ra * ap[1] + rb * bn[1];
    const double my0 = ra * av * ap[0] + rb * bv * bn[0];
    const double mz0 = ra * aw * ap[0] + rb * bw * bn[0];
    const double E0 = 0.5 * (ra * (ap[2] + ta * ap[0]) + rb * (bn[2] + tb * bn[0]));
    if (!(rho0 > 0.0)) return;
    const double U0 = mx0 / rho0, V0 = my0 / rho0, W0 = mz0 / rho0;
    const double T0 = (E0 / rho0 - 0.5 * (U0 * U0 + V0 * V0 + W0 * W0)) / (1.5 * I.R);
    if (!(T0 > 0.0)) return;
    const double p0 = rho0 * I.R * T0;
    const double mu0 = viscosity(I, T0);
    const double tauf = mu0 / p0;
    double Pf;
    if (I.split_mode == 1) {
        Pf = -expm1(-(I.dt / tauf));                 // the flux of Sec. 3.3 at t = dt
    } else {
        if (I.dt <= tauf) return;
        Pf = 1.0 - tauf / I.dt;
    }
    double G[5];
    if (I.flux_mode == 1) {
        G[0] = ra * ap[1] + rb * bn[1];
        G[1] = ra * ap[2] + rb * bn[2];
        G[2] = ra * av * ap[1] + rb * bv * bn[1];
        G[3] = ra * aw * ap[1] + rb * bw * bn[1];
        G[4] = 0.5 * (ra * (ap[3] + ta * ap[1]) + rb * (bn[3] + tb * bn[1]));
    } else {
        G[0] = mx0;
        G[1] = mx0 * U0 + p0;
        G[2] = mx0 * V0;
        G[3] = mx0 * W0;
        G[4] = U0 * (E0 + p0);
    }
    if (aok && bok) {
        const double mue = eps_factor(I.eps_mode, I.dt / tauf) * mu0;
        const double kap = 2.5 * I.R * mue / I.Pr;
        const double inv = 1.0 / I.dx;
        const double sxx = (4.0 / 3.0) * mue * ((gb[1] - ga[1]) * inv);
        const double sxy = mue * ((gb[2] - ga[2]) * inv);
        const double sxz = mue * ((gb[3] - ga[3]) * inv);
        G[1] -= sxx;
        G[2] -= sxy;
        G[3] -= sxz;
        G[4] -= U0 * sxx + V0 * sxy + W0 * sxz + kap * ((gb[4] - ga[4]) * inv);
    }
    for (int k = 0; k < 5; ++k) F[k] = Pf * G[k];
}

}  // namespace duwp

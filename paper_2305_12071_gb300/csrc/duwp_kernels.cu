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
    int64_t k = static_cast<int64_t>(fk);
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
// NTC collisions of one cell (Appendix A), one thread, candidates in order.
// ------------------------------------------------------------------------------------------
template <typename Rec>
__device__ void collide_cell(const InstDev &I, uint32_t id, uint32_t step, Rec *list, int N, double rho_t,
                             double &cmax, int &ncand, int &nacc)
{
    using T = decltype(list[0].xl);
    ncand = 0;
    nacc = 0;
    if (N < 2) return;
    const double rr = (I.ntc_rate == 1) ? rho_t / I.rho_ref : ((static_cast<double>(N) * I.mp) / I.dx) / I.rho_ref;
    const double f = (I.upsilon == 0.0) ? 1.0 : pow(cmax / I.c_ref, -2.0 * I.upsilon);
    const double nsel = I.ntc_A * rr * (static_cast<double>(N) - 1.0) * f * cmax;
    uint32_t w[4];
    draw(I, id, 1u, step, kRound, w);
    int64_t nc = static_cast<int64_t>(floor(nsel + u53(w[0], w[1])));
    if (!(nsel < 1e8)) nc = -1;   // reported by the caller as an overflow; no candidates run
    const double expo = 1.0 - 2.0 * I.upsilon;
    int acc = 0;
    for (int64_t k = 0; k < nc; ++k) {
        draw(I, id, static_cast<uint32_t>(2 * k), step, kCollide, w);
        const uint32_t a = idx32(w[0], static_cast<uint32_t>(N));
        uint32_t b = idx32(w[1], static_cast<uint32_t>(N - 1));
        if (b >= a) ++b;
        Rec A = list[a], B = list[b];
        const double au = A.u, av = A.v, aw = A.w, bu = B.u, bv = B.v, bw = B.w;
        const double d0 = au - bu, d1 = av - bv, d2 = aw - bw;
        const double cr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        if (cr > cmax) cmax = cr;
        const double x = cr / cmax;
        const double prob = (I.upsilon == 0.0) ? x : pow(x, expo);
        if (u53(w[2], w[3]) < prob) {
            uint32_t v[4];
            draw(I, id, static_cast<uint32_t>(2 * k + 1), step, kCollide, v);
            const double ct = 2.0 * u53(v[0], v[1]) - 1.0;
            const double st = sqrt(1.0 - ct * ct);
            const double ph = kTwoPi * u53(v[2], v[3]);
            const double c0 = (cr * st) * cos(ph), c1 = (cr * st) * sin(ph), c2 = cr * ct;
            const double m0 = (au + bu) * 0.5, m1 = (av + bv) * 0.5, m2 = (aw + bw) * 0.5;
            A.u = store_val(m0 + c0 * 0.5, T());
            A.v = store_val(m1 + c1 * 0.5, T());
            A.w = store_val(m2 + c2 * 0.5, T());
            B.u = store_val(m0 - c0 * 0.5, T());
            B.v = store_val(m1 - c1 * 0.5, T());
            B.w = store_val(m2 - c2 * 0.5, T());
            list[a] = A;
            list[b] = B;
            ++acc;
        }
    }
    ncand = static_cast<int>(nc);
    nacc = acc;
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
// Particle kernel
// ------------------------------------------------------------------------------------------
struct CellHdr {
    int b, i, C, ghost, skip;
    int n_in, slots, n_surv, n_new, n_tot;
    int nfb, nfa, fb, fa;
    int64_t Ra, Sa, La, off_out;
    int Rn, Sn, Ln;
    double P, rho_t, cmax;
    double q[5];
    int valid;
    int ncand, nacc;
    int cntL, cntS, cntR;
};

template <typename Rec>
__global__ void __launch_bounds__(512) k_particles(EngineDev E, int rp)
{
    using T = decltype(Rec().xl);
    extern __shared__ __align__(16) unsigned char smraw[];
    Rec *sm = reinterpret_cast<Rec *>(smraw);
    uint8_t *cls = smraw + static_cast<size_t>(E.cell_cap) * sizeof(Rec);
    __shared__ CellHdr H;
    __shared__ int s_g;
    __shared__ uint64_t s_scan[32];
    __shared__ double s_red[32][13];
    __shared__ uint64_t s_run;

    const int wp = 1 - rp;
    const Rec *in = static_cast<const Rec *>(E.buf[rp]);
    Rec *out = static_cast<Rec *>(E.buf[wp]);
    const FarItem<Rec> *fs = static_cast<const FarItem<Rec> *>(E.far_sorted);
    FarItem<Rec> *fa = static_cast<FarItem<Rec> *>(E.far_app);
    const int tid = threadIdx.x, nt = blockDim.x;

    for (;;) {
        if (tid == 0) s_g = atomicAdd(E.ticket, 1);
        __syncthreads();
        const int g = s_g;
        if (g >= E.G) break;

        // ---------------- header (one thread)
        if (tid == 0) {
            H.skip = 0;
            H.b = E.cell_inst[g];
            H.ncand = H.nacc = 0;
            H.cntL = H.cntS = H.cntR = 0;
            H.n_in = H.n_surv = H.n_new = H.n_tot = 0;
            H.nfb = H.nfa = 0;
            H.Rn = H.Sn = H.Ln = 0;
            if (H.b < 0) {
                H.skip = 1;
            } else {
                const InstDev &I = E.inst[H.b];
                H.C = I.C;
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
                    if (H.n_in != E.cnt[g] || H.n_in > E.cell_cap) {
                        set_err(E.err, kErrOverflow);
                        H.skip = 1;
                    }
                }
            }
        }
        __syncthreads();
        if (H.skip) {
            if (tid == 0) {
                E.nL[wp][g] = 0; E.nS[wp][g] = 0; E.nR[wp][g] = 0;
                for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0.0; E.AR[4 * g + k] = 0.0; }
                for (int k = 0; k < 5; ++k) E.Aself[5 * g + k] = 0.0;
                E.ncand[g] = 0; E.nacc[g] = 0; E.nabs[g] = 0; E.nnew[g] = 0;
            }
            __syncthreads();
            continue;
        }
        const InstDev &I = E.inst[H.b];
        const uint32_t step = I.step;
        const uint32_t id = static_cast<uint32_t>(H.i + 1);

        // ---------------- gather the arrived list into shared memory
        const int n_in = H.n_in;
        for (int k = tid; k < n_in; k += nt) {
            int r = k;
            Rec v;
            if (r < H.nfb) { v = fs[H.fb + r].rec; }
            else if ((r -= H.nfb) < H.Rn) { v = ld_rec(in + H.Ra + r); }
            else if ((r -= H.Rn) < H.Sn) { v = ld_rec(in + H.Sa + r); }
            else if ((r -= H.Sn) < H.Ln) { v = ld_rec(in + H.La + r); }
            else { r -= H.Ln; v = fs[H.fa + r].rec; }
            sm[k] = v;
        }
        __syncthreads();

        // ---------------- absorption into the wave with probability P (Eq. p), stable compaction
        int n_surv = n_in;
        if (!H.ghost && H.P > 0.0) {
            const double P = H.P;
            if (tid == 0) s_run = 0;
            __syncthreads();
            for (int base = 0; base < n_in; base += nt) {
                const int k = base + tid;
                Rec v;
                int keep = 0;
                if (k < n_in) {
                    v = sm[k];
                    uint32_t w[4];
                    draw(I, id, static_cast<uint32_t>(k), step, kAbsorb, w);
                    keep = !(u53(w[0], w[1]) < P);
                }
                uint64_t tot;
                const uint64_t pos = block_scan_u64(static_cast<uint64_t>(keep), s_scan, &tot);
                const uint64_t run = s_run;
                __syncthreads();
                if (keep) sm[run + pos] = v;
                __syncthreads();
                if (tid == 0) s_run = run + tot;
                __syncthreads();
            }
            n_surv = static_cast<int>(s_run);
        }

        // ---------------- re-sampling of (1-P) of the wave (Step 2), then collisions (Appendix A)
        if (tid == 0) {
            H.n_surv = n_surv;
            if (!H.ghost) {
                const double rho_w = H.rho_t - static_cast<double>(n_surv) * I.mp_over_dx;
                H.n_new = H.valid ? static_cast<int>(resample_count(I, id, step, H.P, rho_w)) : 0;
            }
            H.n_tot = n_surv + H.n_new;
            if (H.n_tot > H.slots || H.n_tot > E.cell_cap || H.off_out + H.n_tot > E.capacity) {
                set_err(E.err, kErrOverflow);
                H.skip = 1;
            }
        }
        __syncthreads();
        if (H.skip) {
            if (tid == 0) {
                E.nL[wp][g] = 0; E.nS[wp][g] = 0; E.nR[wp][g] = 0;
                for (int k = 0; k < 4; ++k) { E.AL[4 * g + k] = 0.0; E.AR[4 * g + k] = 0.0; }
                for (int k = 0; k < 5; ++k) E.Aself[5 * g + k] = 0.0;
            }
            __syncthreads();
            continue;
        }
        const int n_tot = H.n_tot;
        for (int j = tid; j < H.n_new; j += nt) sm[n_surv + j] = sample_particle<Rec>(I, id, static_cast<uint32_t>(j), step, H.q);
        __syncthreads();
        if (!H.ghost && tid == 0) {
            double cmax = H.cmax;
            int nc = 0, na = 0;
            collide_cell<Rec>(I, id, step, sm, n_tot, H.rho_t, cmax, nc, na);
            if (nc < 0) { set_err(E.err, kErrOverflow); nc = 0; }
            H.ncand = nc;
            H.nacc = na;
            E.cmax[g] = cmax;
        }
        __syncthreads();

        // ---------------- transport and classification (pass A)
        double aL[4] = {0, 0, 0, 0}, aR[4] = {0, 0, 0, 0}, aS[5] = {0, 0, 0, 0, 0};
        int cL = 0, cS = 0, cR = 0;
        const int cell_base = I.cell_base;
        for (int k = tid; k < n_tot; k += nt) {
            Rec v = sm[k];
            const double u0 = v.u;
            T xl = v.xl, uu = v.u;
            bool refl = false;
            const int64_t d = transport(I, H.i, xl, uu, refl);
            v.xl = xl;
            v.u = uu;
            const double u1 = uu, vv = v.v, ww = v.w;
            const double e_pre = 0.5 * (u0 * u0 + vv * vv + ww * ww);
            const double e_post = 0.5 * (u1 * u1 + vv * vv + ww * ww);
            int c;
            if (d < 0) c = 4;
            else if (d == H.i - 1) c = 0;
            else if (d == H.i) c = 1;
            else if (d == H.i + 1) c = 2;
            else c = 3;
            if (c == 1) {
                ++cS;
                if (refl) aS[1] += u1 - u0;
            } else {
                aS[0] -= 1.0; aS[1] -= u0; aS[2] -= vv; aS[3] -= ww; aS[4] -= e_pre;
                if (c == 0) { ++cL; aL[0] += u1; aL[1] += vv; aL[2] += ww; aL[3] += e_post; }
                else if (c == 2) { ++cR; aR[0] += u1; aR[1] += vv; aR[2] += ww; aR[3] += e_post; }
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
            sm[k] = v;
            cls[k] = static_cast<uint8_t>(c);
        }
        // reductions of the class counts and moment sums
        {
            const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
            double vals[13] = {aL[0], aL[1], aL[2], aL[3], aR[0], aR[1], aR[2], aR[3], aS[0], aS[1], aS[2], aS[3], aS[4]};
#pragma unroll
            for (int k = 0; k < 13; ++k) vals[k] = warp_sum(vals[k]);
            int c3[3] = {cL, cS, cR};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c3[k] += __shfl_down_sync(0xffffffffu, c3[k], o);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 13; ++k) s_red[warp][k] = vals[k];
                atomicAdd(&H.cntL, c3[0]);
                atomicAdd(&H.cntS, c3[1]);
                atomicAdd(&H.cntR, c3[2]);
            }
            __syncthreads();
            if (tid < 13) {
                double s = 0.0;
                for (int w = 0; w < nw; ++w) s += s_red[w][tid];
                if (tid < 4) E.AL[4 * g + tid] = s;
                else if (tid < 8) E.AR[4 * g + tid - 4] = s;
                else E.Aself[5 * g + tid - 8] = s;
            }
        }
        __syncthreads();

        // ---------------- stable partition into the cell's output block [L | S | R] (pass B)
        const int nL = H.cntL, nS = H.cntS;
        if (tid == 0) s_run = 0;
        __syncthreads();
        for (int base = 0; base < n_tot; base += nt) {
            const int k = base + tid;
            int c = 5;
            Rec v;
            if (k < n_tot) { c = cls[k]; v = sm[k]; }
            const uint64_t f = (c == 0) ? 1ull : (c == 1) ? (1ull << 21) : (c == 2) ? (1ull << 42) : 0ull;
            uint64_t tot;
            const uint64_t pre = block_scan_u64(f, s_scan, &tot);
            const uint64_t run = s_run;
            if (c <= 2) {
                const uint64_t msk = (1ull << 21) - 1;
                const int sh = 21 * c;
                const int64_t rank = static_cast<int64_t>(((run >> sh) & msk) + ((pre >> sh) & msk));
                const int64_t basec = (c == 0) ? 0 : (c == 1) ? nL : nL + nS;
                st_rec(out + H.off_out + basec + rank, v);
            }
            __syncthreads();
            if (tid == 0) s_run = run + tot;
            __syncthreads();
        }
        if (tid == 0) {
            if (!H.ghost) atomicAdd(&E.inst[H.b].updates, static_cast<unsigned long long>(n_tot));
            E.nL[wp][g] = H.cntL;
            E.nS[wp][g] = H.cntS;
            E.nR[wp][g] = H.cntR;
            E.ncand[g] = H.ncand;
            E.nacc[g] = H.nacc;
            E.nabs[g] = H.n_in - H.n_surv;
            E.nnew[g] = H.n_new;
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
    return sizeof(CellHdr) + 4 + 32 * 8 + 32 * 13 * 8 + 8 + 64;
}

int max_cell_capacity(int fp32)
{
    const size_t limit = 227 * 1024 - static_smem_particles();
    const size_t per = (fp32 ? sizeof(RecF) : sizeof(RecD)) + 1;
    return static_cast<int>((limit - 16) / per);
}

int particles_occupancy(int fp32, int threads, size_t smem)
{
    int n = 0;
    cudaError_t e;
    if (fp32) {
        cudaFuncSetAttribute(k_particles<RecF>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_particles<RecF>, threads, smem);
    } else {
        cudaFuncSetAttribute(k_particles<RecD>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_particles<RecD>, threads, smem);
    }
    if (e != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_particles(const EngineDev &E, int fp32, int rp, int grid, int threads, size_t smem, cudaStream_t s)
{
    if (fp32) k_particles<RecF><<<grid, threads, smem, s>>>(E, rp);
    else k_particles<RecD><<<grid, threads, smem, s>>>(E, rp);
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

/*
 * duwp_oracle.c -- plain, slow, single-threaded FP64 restatement of the direct
 * unified wave-particle (DUWP) time step (Cao, Liu, Yang, Zhong, arXiv 2305.12071).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call this file.  The CUDA
 * library never links it and shares no source with it: the Philox generator,
 * the moment definitions, the NS flux, the collision and streaming arithmetic
 * are all written out again here, from the paper and from the published
 * generator description, in the order the paper gives them.
 *
 * Step of one instance (Sec. 3.4, "Algorithm of DUWP", Steps 1-4):
 *   1. total state  Psi_t = Psi_w + Psi_p  per cell                  (Step 1)
 *   2. per cell: P from Eq. (p); each particle absorbed with prob. P;
 *      (1-P) of the wave mass re-sampled as Maxwellian particles at the
 *      total state (Eq. maxsample); NTC/VHS collisions (Appendix A)  (Step 2)
 *   3. free transport x += xi*dt, particle flux Eq. (fp) as the change of
 *      the per-cell particle moments, wave flux by an NS solver, and the
 *      conservative update Eq. (r1)                                  (Step 3)
 *
 * Points the paper leaves open are each taken one way and marked "reading"
 * where they are implemented: the wave-flux scheme of Step 3 (Sec. 3.3 names
 * only "N-S solvers"), its weight (Eq. p applied at the interface state), the
 * rounding of particle counts (Step 2), the boundary handling (Sec. 4 gives
 * none) and the counter layout of the random numbers (the paper draws them
 * without specifying a generator).
 *
 * Precision: all arithmetic is FP64.  With `fp32 = 1` the particle record
 * (cell-local position and velocity) is STORED in single precision: every
 * value written to a particle is rounded to float, and the free-transport
 * position update (the one floating-point result that decides an integer,
 * the new cell) is taken in single precision with one fused multiply-add,
 * the way the single-precision particle store evaluates it.
 *
 * Parity pins: tests/test_oracle_*.py check this file against closed forms,
 * conservation identities, brute force and published generator vectors.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -o liboracle.so duwp_oracle.c -lm
 * (-ffp-contract=off: no silent fused multiply-adds; the fused ones are explicit.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_PI 3.14159265358979323846
#define ORA_TWO_PI 6.283185307179586

/* ------------------------------------------------------------------------- */
/* Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,         */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 5):              */
/* 10 rounds of two 32x32->64 multiplies with a key schedule bumped by the     */
/* Weyl constants between rounds.                                              */
/* ------------------------------------------------------------------------- */
void ora_philox(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 53-bit uniform in [0,1) from two words: the top 32 bits from a, 21 from b. */
double ora_u53(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)a << 21) ^ (uint64_t)(b >> 11);
    return (double)m * (1.0 / 9007199254740992.0);
}

/* Draw purposes (fourth counter word).  Reading: the RNG layout is not in the
 * paper; every random number is keyed by (id, sub, step, purpose). */
enum { ORA_ABSORB = 1, ORA_ROUND = 2, ORA_SAMPLE = 3, ORA_COLLIDE = 4 };

typedef struct { uint32_t k0, k1; } ora_key;

static void draw(ora_key key, uint32_t id, uint32_t sub, uint32_t step, uint32_t purpose,
                 uint32_t w[4])
{
    uint32_t c[4] = { id, sub, step, purpose };
    ora_philox(key.k0, key.k1, c, w);
}

/* Unbiased-enough integer pick in [0,n) by the multiply-shift map of a 32-bit word. */
static uint32_t pick(uint32_t w, uint32_t n) { return (uint32_t)(((uint64_t)w * n) >> 32); }

/* Pair of distinct indices in [0,N) (N >= 2): a uniform, b uniform over the others. */
void ora_pick_pair(uint32_t w0, uint32_t w1, uint32_t N, uint32_t *a, uint32_t *b)
{
    uint32_t ia = pick(w0, N);
    uint32_t ib = pick(w1, N - 1u);
    if (ib >= ia) ib += 1u;
    *a = ia; *b = ib;
}

/* ------------------------------------------------------------------------- */
/* Problem description (the paper's problem statement: gas and VHS constants, */
/* mesh, Kn, time step, boundary states; Sec. 4 and Appendix A).              */
/* ------------------------------------------------------------------------- */
typedef struct { double rho, u, v, w, T; } ora_state;

enum { ORA_BC_INOUT = 0, ORA_BC_SPECULAR = 1, ORA_BC_PERIODIC = 2, ORA_BC_VACUUM = 3 };
enum { ORA_EPS1 = 0, ORA_EPS12 = 1, ORA_EPS0 = 2, ORA_EPS_AVG = 3 };
enum { ORA_FLUX_GKS_EQ = 0, ORA_FLUX_KFVS = 1 };
enum { ORA_NTC_PARTICLE = 0, ORA_NTC_TOTAL = 1 };
enum { ORA_RESAMPLE_MAXWELL = 0, ORA_RESAMPLE_CE = 1 };
enum { ORA_SPLIT_P = 0, ORA_SPLIT_QMC = 1 };
enum { ORA_RECON_FIRST = 0, ORA_RECON_VANLEER = 1 };

typedef struct {
    double gamma, Pr, R;
    double omega, alpha;
    double rho_ref, T_ref, Kn, L_ref;
    double x_min, x_max;
    int32_t n_cells;
    double dt, cfl;
    ora_state left, right;
    double x_split;
    int32_t bc_left, bc_right;
    double ppc_ref;
    int32_t fp32, eps_mode, flux_mode, ntc_rate;
    uint64_t seed;
    int32_t avg_start;
    int32_t resample_mode;
    int32_t split_mode;
    int32_t recon_mode;
} ora_params;

typedef struct {
    double dx, dt, dtdx, mp, dx_over_mp, mp_over_dx;
    double beta, lambda_ref, mu_ref, p_ref, upsilon, c_ref, ntc_A;
    float dtdx_f;
} ora_consts;

/* beta of the mean-free-path relation, Eq. (lambda), first form (Sec. 4.1). */
double ora_beta(double omega, double alpha)
{
    return 5.0 * (alpha + 1.0) * (alpha + 2.0) / (4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega));
}

/* c_{r,ref} = sqrt(2 k T_ref / m_r) / Gamma(2.5 - omega)^{0.5/upsilon}, with k = mR and
 * m_r = m/2, so 2kT_ref/m_r = 4 R T_ref (Appendix A).  HS (upsilon = 0) needs none. */
double ora_c_ref(double omega, double R, double T_ref)
{
    double ups = omega - 0.5;
    if (ups == 0.0) return sqrt(4.0 * R * T_ref);
    return sqrt(4.0 * R * T_ref) / pow(tgamma(2.5 - omega), 0.5 / ups);
}

static double smax_of(const ora_state *s, double R)
{
    return fabs(s->u) + 3.0 * sqrt(2.0 * R * s->T);
}

static void derive(const ora_params *p, ora_consts *c)
{
    c->dx = (p->x_max - p->x_min) / (double)p->n_cells;
    c->beta = ora_beta(p->omega, p->alpha);
    c->lambda_ref = p->Kn * p->L_ref;
    c->p_ref = p->rho_ref * p->R * p->T_ref;
    /* Eq. (lambda) solved for mu at the reference state. */
    c->mu_ref = c->beta * c->lambda_ref * c->p_ref * sqrt(2.0 * ORA_PI / (p->R * p->T_ref));
    c->mp = p->rho_ref * c->dx / p->ppc_ref;
    c->dx_over_mp = c->dx / c->mp;
    c->mp_over_dx = c->mp / c->dx;
    if (p->dt > 0.0) {
        c->dt = p->dt;
    } else {
        /* reading: one global dt fixed at start from the CFL number and the
         * fastest initial state (|U| + 3 sqrt(2RT)). */
        double s = smax_of(&p->left, p->R);
        double s2 = smax_of(&p->right, p->R);
        if (s2 > s) s = s2;
        c->dt = p->cfl * c->dx / s;
    }
    c->dtdx = c->dt / c->dx;
    c->dtdx_f = (float)c->dtdx;
    c->upsilon = p->omega - 0.5;
    c->c_ref = ora_c_ref(p->omega, p->R, p->T_ref);
    c->ntc_A = c->dt / (2.0 * sqrt(2.0) * c->lambda_ref);
}

/* ------------------------------------------------------------------------- */
/* Macroscopic quantities (Sec. 2): Psi = (rho, rho U, rho V, rho W, rho E),  */
/* rho E = 1/2 rho |U|^2 + 3/2 rho R T for a monatomic gas (D = 0).            */
/* ------------------------------------------------------------------------- */
typedef struct { double rho, u, v, w, T; int valid; } ora_prim;

static void cons_of_state(const ora_state *s, double R, double psi[5])
{
    psi[0] = s->rho;
    psi[1] = s->rho * s->u;
    psi[2] = s->rho * s->v;
    psi[3] = s->rho * s->w;
    psi[4] = 0.5 * s->rho * (s->u * s->u + s->v * s->v + s->w * s->w) + 1.5 * s->rho * R * s->T;
}

static ora_prim prim_of_cons(const double psi[5], double R)
{
    ora_prim q;
    q.rho = psi[0];
    q.valid = 0;
    q.u = q.v = q.w = q.T = 0.0;
    if (!(q.rho > 0.0)) return q;
    q.u = psi[1] / q.rho;
    q.v = psi[2] / q.rho;
    q.w = psi[3] / q.rho;
    double e = psi[4] / q.rho - 0.5 * (q.u * q.u + q.v * q.v + q.w * q.w);
    q.T = e / (1.5 * R);
    q.valid = (q.T > 0.0) && isfinite(q.T) && isfinite(q.u) && isfinite(q.v) && isfinite(q.w);
    return q;
}

static double mu_of_T(const ora_params *p, const ora_consts *c, double T)
{
    return c->mu_ref * pow(T / p->T_ref, p->omega);
}

/* Absorption fraction, Eq. (p): P = 0 for dt <= tau, 1 - tau/dt otherwise; tau = mu/p.
 * split_mode QMC (Sec. 3.2, the multi-scale Boltzmann equation solved by quantified model
 * competition): a particle collides during dt, and joins the wave, with probability
 * 1 - exp(-dt/tau). */
static double pfrac(const ora_params *p, const ora_consts *c, const ora_prim *q)
{
    if (!q->valid) return 0.0;
    double tau = mu_of_T(p, c, q->T) / (q->rho * p->R * q->T);
    if (p->split_mode == ORA_SPLIT_QMC) return -expm1(-(c->dt / tau));
    if (c->dt <= tau) return 0.0;
    return 1.0 - tau / c->dt;
}

/* Viscosity correction factors of Sec. 3.3 as functions of x = dt/tau:
 * eps1 (Eq. vp1) = 1 - x e^{-x}/(1-e^{-x}) = 1 - x/(e^x - 1); eps12 = x/(2+x); eps0 = 1;
 * time-averaged eps (Eq. vp) = [-2(1-e^{-x}) + x(1+e^{-x})] / [x - (1-e^{-x})]. */
double ora_eps(int mode, double x)
{
    if (mode == ORA_EPS0) return 1.0;
    if (mode == ORA_EPS12) return x / (2.0 + x);
    if (mode == ORA_EPS_AVG) {
        double a = -expm1(-x);          /* 1 - e^{-x} */
        double b = 1.0 + exp(-x);       /* 1 + e^{-x} */
        return (-2.0 * a + x * b) / (x - a);
    }
    double d = expm1(x);                 /* e^x - 1, overflows to inf for large x: eps -> 1 */
    return 1.0 - x / d;
}

/* Moments of the half-Maxwellian in the normal velocity u (unit density):
 * Mp[n] = <u^n> over u > 0, Mm[n] over u < 0, with lam = 1/(2RT).
 * <u^0> = erfc(-+sqrt(lam) U)/2, <u^1> = U<u^0> +- e^{-lam U^2}/(2 sqrt(pi lam)),
 * <u^{n+1}> = U <u^n> + n/(2 lam) <u^{n-1}>. */
void ora_half_moments(double U, double lam, double Mp[4], double Mm[4])
{
    double sl = sqrt(lam);
    Mp[0] = 0.5 * erfc(-sl * U);
    Mm[0] = 0.5 * erfc(sl * U);
    double e = 0.5 * exp(-lam * U * U) / sqrt(ORA_PI * lam);
    Mp[1] = U * Mp[0] + e;
    Mm[1] = U * Mm[0] - e;
    for (int n = 1; n <= 2; ++n) {
        Mp[n + 1] = U * Mp[n] + (double)n * Mp[n - 1] / (2.0 * lam);
        Mm[n + 1] = U * Mm[n] + (double)n * Mm[n - 1] / (2.0 * lam);
    }
}

/* Wave flux across one interface (Step 3, "calculated by N-S solvers"; Sec. 3.3, Eq. ce2
 * evaluated at t = dt with eps1 of Eq. vp1).  Reading: first-order states; the
 * interface equilibrium W0 is built from the right-going half of the left
 * Maxwellian and the left-going half of the right one (GKS_EQ), or the flux is the
 * split kinetic flux of the two halves (KFVS); the NS viscous and heat-flux terms use
 * mu_e = eps * mu(T0) and one-sided differences of the neighbouring cell states (GL, GR: the
 * cell states, also when L and R are reconstructed interface states); the
 * whole wave flux is weighted by P_f = max(0, 1 - tau_f/dt) at the interface state
 * (split_mode QMC: by 1 - exp(-dt/tau_f), the weight of Sec. 3.3's flux at t = dt).
 * Returns the flux per unit area (mass, x/y/z momentum, energy). */
static void wave_flux(const ora_params *p, const ora_consts *c, const ora_prim *L, const ora_prim *Rr,
                      const ora_prim *GL, const ora_prim *GR, int viscous_ok, double F[5])
{
    for (int k = 0; k < 5; ++k) F[k] = 0.0;
    double MpL[4] = { 0, 0, 0, 0 }, MmL[4] = { 0, 0, 0, 0 };
    double MpR[4] = { 0, 0, 0, 0 }, MmR[4] = { 0, 0, 0, 0 };
    double lamL = 0.0, lamR = 0.0;
    if (L->valid) { lamL = 1.0 / (2.0 * p->R * L->T); ora_half_moments(L->u, lamL, MpL, MmL); }
    if (Rr->valid) { lamR = 1.0 / (2.0 * p->R * Rr->T); ora_half_moments(Rr->u, lamR, MpR, MmR); }
    double rL = L->valid ? L->rho : 0.0, rR = Rr->valid ? Rr->rho : 0.0;
    double tL = L->valid ? (L->v * L->v + L->w * L->w + 1.0 / lamL) : 0.0;
    double tR = Rr->valid ? (Rr->v * Rr->v + Rr->w * Rr->w + 1.0 / lamR) : 0.0;

    /* interface equilibrium state W0 (conservative) */
    double rho0 = rL * MpL[0] + rR * MmR[0];
    double m0 = rL * MpL[1] + rR * MmR[1];
    double mv0 = rL * L->v * MpL[0] + rR * Rr->v * MmR[0];
    double mw0 = rL * L->w * MpL[0] + rR * Rr->w * MmR[0];
    double E0 = 0.5 * (rL * (MpL[2] + tL * MpL[0]) + rR * (MmR[2] + tR * MmR[0]));
    if (!(rho0 > 0.0)) return;
    double U0 = m0 / rho0, V0 = mv0 / rho0, W0 = mw0 / rho0;
    double T0 = (E0 / rho0 - 0.5 * (U0 * U0 + V0 * V0 + W0 * W0)) / (1.5 * p->R);
    if (!(T0 > 0.0)) return;
    double p0 = rho0 * p->R * T0;
    double mu0 = mu_of_T(p, c, T0);
    double tauf = mu0 / p0;
    double Pf;
    if (p->split_mode == ORA_SPLIT_QMC) {
        Pf = -expm1(-(c->dt / tauf));          /* the flux of Sec. 3.3 at t = dt */
    } else {
        if (c->dt <= tauf) return;             /* P_f = 0: no wave flux (DSMC regime) */
        Pf = 1.0 - tauf / c->dt;
    }

    double Fe[5];
    if (p->flux_mode == ORA_FLUX_KFVS) {
        Fe[0] = rL * MpL[1] + rR * MmR[1];
        Fe[1] = rL * MpL[2] + rR * MmR[2];
        Fe[2] = rL * L->v * MpL[1] + rR * Rr->v * MmR[1];
        Fe[3] = rL * L->w * MpL[1] + rR * Rr->w * MmR[1];
        Fe[4] = 0.5 * (rL * (MpL[3] + tL * MpL[1]) + rR * (MmR[3] + tR * MmR[1]));
    } else {
        /* Euler flux of the interface equilibrium g0 */
        Fe[0] = m0;
        Fe[1] = m0 * U0 + p0;
        Fe[2] = m0 * V0;
        Fe[3] = m0 * W0;
        Fe[4] = U0 * (E0 + p0);
    }
    if (viscous_ok && GL->valid && GR->valid) {
        double x = c->dt / tauf;
        double eps = ora_eps(p->eps_mode, x);
        double mue = eps * mu0;
        double kape = 2.5 * p->R * mue / p->Pr;
        double dU = (GR->u - GL->u) / c->dx;
        double dV = (GR->v - GL->v) / c->dx;
        double dW = (GR->w - GL->w) / c->dx;
        double dT = (GR->T - GL->T) / c->dx;
        double txx = (4.0 / 3.0) * mue * dU;
        double txy = mue * dV;
        double txz = mue * dW;
        Fe[1] -= txx;
        Fe[2] -= txy;
        Fe[3] -= txz;
        Fe[4] -= U0 * txx + V0 * txy + W0 * txz + kape * dT;
    }
    for (int k = 0; k < 5; ++k) F[k] = Pf * Fe[k];
}

/* exported for the pin tests: flux of two primitive states */
void ora_wave_flux(const ora_params *p, const double WL[5], const double WR[5], int viscous_ok, double F[5])
{
    ora_consts c;
    derive(p, &c);
    ora_prim L = { WL[0], WL[1], WL[2], WL[3], WL[4], 0 }, Rr = { WR[0], WR[1], WR[2], WR[3], WR[4], 0 };
    L.valid = (L.rho > 0.0 && L.T > 0.0);
    Rr.valid = (Rr.rho > 0.0 && Rr.T > 0.0);
    wave_flux(p, &c, &L, &Rr, &L, &Rr, viscous_ok, F);
}

/* Second-order wave reconstruction (recon_mode = VANLEER; reading): per primitive variable
 * (rho, U, V, W, T) the van Leer limited slope s = 2 dl dr / (dl + dr) where the one-sided
 * differences dl, dr have the same sign, else 0; the interface between cells 0 and 1 sees
 * W0 + s0/2 on the left and W1 - s1/2 on the right.  use0 / use1 = 0: that cell's slope is 0 (a
 * reservoir or mirror cell, or an unusable neighbour).  If a reconstructed state has rho <= 0 or
 * T <= 0 the interface keeps the cell states. */
static void vl_slopes(const ora_prim *a, const ora_prim *b, const ora_prim *cc, double s[5])
{
    const double qa[5] = { a->rho, a->u, a->v, a->w, a->T };
    const double qb[5] = { b->rho, b->u, b->v, b->w, b->T };
    const double qc[5] = { cc->rho, cc->u, cc->v, cc->w, cc->T };
    for (int k = 0; k < 5; ++k) {
        double dl = qb[k] - qa[k], dr = qc[k] - qb[k];
        s[k] = (dl * dr > 0.0) ? (2.0 * dl * dr) / (dl + dr) : 0.0;
    }
}

static void recon_pair(const ora_prim *Wm, const ora_prim *W0, const ora_prim *W1, const ora_prim *W2, int use0,
                       int use1, ora_prim *LR, ora_prim *RR)
{
    *LR = *W0;
    *RR = *W1;
    if (!W0->valid || !W1->valid) return;
    double s0[5] = { 0, 0, 0, 0, 0 }, s1[5] = { 0, 0, 0, 0, 0 };
    if (use0 && Wm->valid) vl_slopes(Wm, W0, W1, s0);
    if (use1 && W2->valid) vl_slopes(W0, W1, W2, s1);
    ora_prim a = *W0, b = *W1;
    a.rho = W0->rho + 0.5 * s0[0]; a.u = W0->u + 0.5 * s0[1]; a.v = W0->v + 0.5 * s0[2];
    a.w = W0->w + 0.5 * s0[3]; a.T = W0->T + 0.5 * s0[4];
    b.rho = W1->rho - 0.5 * s1[0]; b.u = W1->u - 0.5 * s1[1]; b.v = W1->v - 0.5 * s1[2];
    b.w = W1->w - 0.5 * s1[3]; b.T = W1->T - 0.5 * s1[4];
    if (a.rho > 0.0 && a.T > 0.0 && b.rho > 0.0 && b.T > 0.0) { *LR = a; *RR = b; }
}

/* exported for the pin tests: the reconstructed interface states between W0 and W1 */
void ora_recon_pair(const double Wm5[5], const double W05[5], const double W15[5], const double W25[5],
                    double WL[5], double WR[5])
{
    ora_prim q[4];
    const double *src[4] = { Wm5, W05, W15, W25 };
    for (int j = 0; j < 4; ++j) {
        q[j].rho = src[j][0]; q[j].u = src[j][1]; q[j].v = src[j][2]; q[j].w = src[j][3]; q[j].T = src[j][4];
        q[j].valid = (q[j].rho > 0.0 && q[j].T > 0.0);
    }
    ora_prim a, b;
    recon_pair(&q[0], &q[1], &q[2], &q[3], 1, 1, &a, &b);
    WL[0] = a.rho; WL[1] = a.u; WL[2] = a.v; WL[3] = a.w; WL[4] = a.T;
    WR[0] = b.rho; WR[1] = b.u; WR[2] = b.v; WR[3] = b.w; WR[4] = b.T;
}

/* ------------------------------------------------------------------------- */
/* Particles                                                                   */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t cell; double xl, u, v, w; } opart;

static double st(const ora_params *p, double x) { return p->fp32 ? (double)(float)x : x; }

/* The moments phi = (1, xi, |xi|^2/2) of one particle (Sec. 2), mass factor applied by caller. */
static void add_phi(double acc[5], const opart *q)
{
    acc[0] += 1.0;
    acc[1] += q->u;
    acc[2] += q->v;
    acc[3] += q->w;
    acc[4] += 0.5 * (q->u * q->u + q->v * q->v + q->w * q->w);
}

/* Chapman-Enskog correction of the re-sampled particles (resample_mode = CE; reading of "the
 * local equilibrium with its NS correction"): the density f_M (1 + Gamma_1) whose pressure tensor
 * is p delta_ij + sigma_ij and whose heat flux is q, to first order in the gradients:
 *   Gamma = 1 + sigma_ij c_i c_j / (2 p R T) + (q . c / (p R T)) (c^2 / (5 R T) - 1),
 * c = xi - U.  With the 1D NS stress and heat flux of the wave (mu_e = eps mu, as in its flux):
 *   sigma_xx = -(4/3) mu_e dU/dx, sigma_yy = sigma_zz = (2/3) mu_e dU/dx, sigma_xy = -mu_e dV/dx,
 *   sigma_xz = -mu_e dW/dx, q_x = -kappa_e dT/dx, kappa_e = (5/2) R mu_e / Pr,
 * gradients by central differences of the neighbouring cell states.  Sampled by acceptance-
 * rejection against the Maxwellian (Garcia and Alder, J. Comput. Phys. 140, 1998): accept with
 * probability Gamma / A, A = 1 + 30 B, B the largest of |sigma_ij| / p and 2 |q_x| / (p sqrt(2RT)).
 * Where B > 1/4 the first-order expansion is out of its range and the Maxwellian is kept. */
#define ORA_CE_ATTEMPTS 64
#define ORA_CE_BMAX 0.25

typedef struct {
    int on;
    double U[3], RT, prt, A;
    double sxx, syy, sxy, sxz, qx;
} ora_ce;

static ora_ce ce_factor(const ora_params *p, const ora_consts *c, const ora_prim *Wm, const ora_prim *W0,
                        const ora_prim *Wp)
{
    ora_ce f;
    memset(&f, 0, sizeof f);
    if (!W0->valid) return f;
    const ora_prim *a = Wm->valid ? Wm : W0, *b = Wp->valid ? Wp : W0;   /* missing neighbour: own state */
    double inv = 1.0 / (2.0 * c->dx);
    double dU = (b->u - a->u) * inv, dV = (b->v - a->v) * inv, dW = (b->w - a->w) * inv, dT = (b->T - a->T) * inv;
    double RT = p->R * W0->T;
    double p0 = W0->rho * RT;
    double mu = mu_of_T(p, c, W0->T);
    double mue = ora_eps(p->eps_mode, c->dt / (mu / p0)) * mu;
    double kap = 2.5 * p->R * mue / p->Pr;
    f.sxx = -(4.0 / 3.0) * mue * dU;
    f.syy = (2.0 / 3.0) * mue * dU;
    f.sxy = -mue * dV;
    f.sxz = -mue * dW;
    f.qx = -kap * dT;
    double B = fmax(fmax(fabs(f.sxx), fabs(f.syy)), fmax(fabs(f.sxy), fabs(f.sxz))) / p0;
    B = fmax(B, 2.0 * fabs(f.qx) / (p0 * sqrt(2.0 * RT)));
    if (!(B <= ORA_CE_BMAX)) return f;
    f.on = 1;
    f.U[0] = W0->u; f.U[1] = W0->v; f.U[2] = W0->w;
    f.RT = RT;
    f.prt = p0 * RT;
    f.A = 1.0 + 30.0 * B;
    return f;
}

static double ce_gamma(const ora_ce *f, const double xi[3])
{
    double cx = xi[0] - f->U[0], cy = xi[1] - f->U[1], cz = xi[2] - f->U[2];
    double c2 = cx * cx + cy * cy + cz * cz;
    double s = f->sxx * cx * cx + f->syy * (cy * cy + cz * cz) + 2.0 * (f->sxy * cx * cy + f->sxz * cx * cz);
    return 1.0 + s / (2.0 * f->prt) + (f->qx * cx / f->prt) * (c2 / (5.0 * f->RT) - 1.0);
}

/* Maxwellian velocities at (U, V, W, T) from words w[0..7], Eq. (maxsample), by the Box-Muller
 * transform (Box and Muller, Ann. Math. Stat. 29, 1958): a uniform angle 2 pi r1 and the radius
 * sqrt(2RT) sqrt(-ln r2) give two independent components, the cosine and the sine; the third takes
 * a second pair of its own and its cosine:
 *   xi_x = U + (sqrt(2RT) cos(2 pi r1)) sqrt(-ln r2),  xi_y = V + (sqrt(2RT) sin(2 pi r1)) sqrt(-ln r2),
 *   xi_z = W + (sqrt(2RT) cos(2 pi r3)) sqrt(-ln r4),
 * r1 = u53(w0, w1), r2 = 1 - u53(w2, w3), r3 = u53(w4, w5), r4 = 1 - u53(w6, w7). */
static void maxwell_xi(const ora_params *p, const ora_prim *q, const uint32_t *w, double xi[3])
{
    double sq = sqrt(2.0 * p->R * q->T);
    double r1 = ora_u53(w[0], w[1]);
    double r2 = 1.0 - ora_u53(w[2], w[3]);
    double r3 = ora_u53(w[4], w[5]);
    double r4 = 1.0 - ora_u53(w[6], w[7]);
    double rad = sqrt(-log(r2));
    xi[0] = q->u + (sq * cos(ORA_TWO_PI * r1)) * rad;
    xi[1] = q->v + (sq * sin(ORA_TWO_PI * r1)) * rad;
    xi[2] = q->w + (sq * cos(ORA_TWO_PI * r3)) * sqrt(-log(r4));
}

/* Sample j of a cell at state q, Eq. (maxsample); position uniform in the cell (reading).  Words of
 * the counters (id, 4j..4j+2, step, SAMPLE): 0-1 position, 2-9 velocities, 10-11 the acceptance
 * draw of the Chapman-Enskog correction (ce != NULL and on); its attempt a > 0 draws the counters
 * (id, 4j..4j+2, step, SAMPLE + 8a).  After ORA_CE_ATTEMPTS rejections the first Maxwellian
 * candidate is kept. */
static void sample_particle(const ora_params *p, ora_key key, uint32_t id, uint32_t j, uint32_t step,
                            const ora_prim *q, const ora_ce *ce, opart *out)
{
    uint32_t w[12];
    for (uint32_t t = 0; t < 3; ++t) draw(key, id, 4u * j + t, step, ORA_SAMPLE, w + 4 * t);
    double xi[3];
    maxwell_xi(p, q, w + 2, xi);
    if (ce && ce->on) {
        double xi0[3] = { xi[0], xi[1], xi[2] };
        int accepted = 0;
        for (uint32_t a = 0; a < ORA_CE_ATTEMPTS; ++a) {
            if (a > 0) {
                for (uint32_t t = 0; t < 3; ++t) draw(key, id, 4u * j + t, step, ORA_SAMPLE + 8u * a, w + 4 * t);
                maxwell_xi(p, q, w + 2, xi);
            }
            if (ora_u53(w[10], w[11]) * ce->A < ce_gamma(ce, xi)) { accepted = 1; break; }
        }
        if (!accepted) { xi[0] = xi0[0]; xi[1] = xi0[1]; xi[2] = xi0[2]; }
        /* the position always comes from the first attempt's words */
        for (uint32_t t = 0; t < 1; ++t) draw(key, id, 4u * j + t, step, ORA_SAMPLE, w + 4 * t);
    }
    double xl = ora_u53(w[0], w[1]);
    if (p->fp32) {
        float xf = (float)xl;
        if (xf >= 1.0f) xf = 0x1.fffffep-1f;
        xl = (double)xf;
    }
    out->xl = xl;
    out->u = st(p, xi[0]);
    out->v = st(p, xi[1]);
    out->w = st(p, xi[2]);
}

/* Isotropic VHS post-collision velocities for equal masses (Appendix A):
 * cos(theta) = 2 r1 - 1, phi = 2 pi r2, xi_r' = c_r (sin cos, sin sin, cos),
 * xi_a' = xi_m + xi_r'/2, xi_b' = xi_m - xi_r'/2, xi_m = (xi_a + xi_b)/2
 * (primes: post-collision values). */
void ora_scatter(double r1, double r2, double a[3], double b[3])
{
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    double cr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    double ct = 2.0 * r1 - 1.0;
    double stt = sqrt(1.0 - ct * ct);
    double ph = ORA_TWO_PI * r2;
    double c0 = (cr * stt) * cos(ph), c1 = (cr * stt) * sin(ph), c2 = cr * ct;
    double m0 = (a[0] + b[0]) * 0.5, m1 = (a[1] + b[1]) * 0.5, m2 = (a[2] + b[2]) * 0.5;
    a[0] = m0 + c0 * 0.5; a[1] = m1 + c1 * 0.5; a[2] = m2 + c2 * 0.5;
    b[0] = m0 - c0 * 0.5; b[1] = m1 - c1 * 0.5; b[2] = m2 - c2 * 0.5;
}

/* NTC candidate count before rounding, nondimensional form of Appendix A:
 * (1/(2 sqrt2 lambda_ref)) (rho/rho_ref) (N-1) dt (c_max/c_ref)^{-2 upsilon} c_max. */
static double ntc_nsel(const ora_consts *c, double rho_ratio, double N, double cmax)
{
    double f = (c->upsilon == 0.0) ? 1.0 : pow(cmax / c->c_ref, -2.0 * c->upsilon);
    return c->ntc_A * rho_ratio * (N - 1.0) * f * cmax;
}

double ora_ntc_nsel(const ora_params *p, double rho_ratio, double N, double cmax)
{
    ora_consts c;
    derive(p, &c);
    return ntc_nsel(&c, rho_ratio, N, cmax);
}

/* Acceptance probability sigma_T c_r / (sigma_T c_r)_max = (c_r/c_max)^{1 - 2 upsilon}. */
static double accept_prob(const ora_consts *c, double cr, double cmax)
{
    double x = cr / cmax;
    if (c->upsilon == 0.0) return x;
    return pow(x, 1.0 - 2.0 * c->upsilon);
}

/* Test hook: the Chapman-Enskog coefficients of a cell with states Wm | W0 | Wp (rho, u, v, w, T
 * each; all valid) and n samples j = 0..n-1 of that cell (counters (id, 4j.., step, ...) of the key
 * (k0, k1)), velocities into xi (n x 3).  coef = (on, sigma_xx, sigma_yy, sigma_xy, sigma_xz, q_x, A). */
void ora_ce_sample(const ora_params *p, const double Wm5[5], const double W05[5], const double Wp5[5],
                   uint32_t k0, uint32_t k1, uint32_t id, uint32_t step, int64_t n, double *xi, double coef[7])
{
    ora_consts c;
    derive(p, &c);
    ora_prim Wm = { Wm5[0], Wm5[1], Wm5[2], Wm5[3], Wm5[4], 1 }, W0 = { W05[0], W05[1], W05[2], W05[3], W05[4], 1 },
             Wp = { Wp5[0], Wp5[1], Wp5[2], Wp5[3], Wp5[4], 1 };
    ora_ce ce = ce_factor(p, &c, &Wm, &W0, &Wp);
    coef[0] = ce.on; coef[1] = ce.sxx; coef[2] = ce.syy; coef[3] = ce.sxy; coef[4] = ce.sxz; coef[5] = ce.qx; coef[6] = ce.A;
    ora_key key = { k0, k1 };
    for (int64_t j = 0; j < n; ++j) {
        opart q;
        sample_particle(p, key, id, (uint32_t)j, step, &W0, &ce, &q);
        xi[3 * j] = q.u; xi[3 * j + 1] = q.v; xi[3 * j + 2] = q.w;
    }
}

/* ------------------------------------------------------------------------- */
/* Instance                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    ora_params p;
    ora_consts c;
    ora_key key;
    int32_t C;
    double *psi;      /* C x 5, total state Psi_t */
    double *avg;      /* C x 5, time-averaged Psi_t */
    int64_t navg;
    double *cmax;     /* C, NTC majorant c_r,max per cell */
    opart *parts;     /* sorted by cell, stable */
    int64_t np, cap;
    uint32_t step;
    /* last-step diagnostics per cell */
    int32_t *ncand, *nacc, *nabs, *nnew;
    int64_t nfar;      /* particles that moved two or more cells (or wrapped) in the last step */
    double *last_flux; /* (C+1) x 5 */
    double *pre_m, *post_m; /* C x 5, particle moment sums of the last step (unscaled) */
    opart *lastpre;   /* pre-transport array of the last step (source cell in .cell) */
    int64_t *lastdest; /* destination cell of each entry, -1 = left the domain */
    int64_t nlastpre;
    /* owned cell range [c0, c1): the whole domain, or one part of a domain decomposition (the
     * other cells' states are only read, as the neighbours of the owned ones) */
    int32_t c0, c1;
    double *F;        /* (C+1) x 5 wave flux of the current step (faces c0..c1) */
    int phase;        /* 1 between the two halves of a step */
} ora_inst;

static int grow(ora_inst *h, opart **arr, int64_t *cap, int64_t need)
{
    if (need <= *cap) return 0;
    int64_t nc = *cap ? *cap : 1024;
    while (nc < need) nc *= 2;
    opart *na = (opart *)realloc(*arr, (size_t)nc * sizeof(opart));
    if (!na) return -1;
    *arr = na;
    *cap = nc;
    (void)h;
    return 0;
}

static ora_prim ghost_prim(const ora_inst *h, int side, const ora_prim *inner)
{
    const ora_params *p = &h->p;
    int bc = side ? p->bc_right : p->bc_left;
    ora_prim g;
    memset(&g, 0, sizeof g);
    if (bc == ORA_BC_INOUT) {
        const ora_state *s = side ? &p->right : &p->left;
        g.rho = s->rho; g.u = s->u; g.v = s->v; g.w = s->w; g.T = s->T;
        g.valid = (g.rho > 0.0 && g.T > 0.0);
    } else if (bc == ORA_BC_SPECULAR) {
        g = *inner;
        g.u = -inner->u;
    } else if (bc == ORA_BC_VACUUM) {
        g.valid = 0;
    }
    return g;
}

void *ora_create(const ora_params *p)
{
    if (p->n_cells < 1 || !(p->x_max > p->x_min) || !(p->ppc_ref > 0.0) || !(p->Kn > 0.0)) return NULL;
    if ((p->bc_left == ORA_BC_PERIODIC) != (p->bc_right == ORA_BC_PERIODIC)) return NULL;
    ora_inst *h = (ora_inst *)calloc(1, sizeof(ora_inst));
    if (!h) return NULL;
    h->p = *p;
    derive(p, &h->c);
    h->key.k0 = (uint32_t)(p->seed & 0xffffffffu);
    h->key.k1 = (uint32_t)(p->seed >> 32);
    h->C = p->n_cells;
    int32_t C = h->C;
    h->psi = (double *)calloc((size_t)C * 5, sizeof(double));
    h->avg = (double *)calloc((size_t)C * 5, sizeof(double));
    h->cmax = (double *)calloc((size_t)C, sizeof(double));
    h->ncand = (int32_t *)calloc((size_t)C, sizeof(int32_t));
    h->nacc = (int32_t *)calloc((size_t)C, sizeof(int32_t));
    h->nabs = (int32_t *)calloc((size_t)C, sizeof(int32_t));
    h->nnew = (int32_t *)calloc((size_t)C, sizeof(int32_t));
    h->last_flux = (double *)calloc((size_t)(C + 1) * 5, sizeof(double));
    h->pre_m = (double *)calloc((size_t)C * 5, sizeof(double));
    h->post_m = (double *)calloc((size_t)C * 5, sizeof(double));
    h->F = (double *)calloc((size_t)(C + 1) * 5, sizeof(double));
    h->c0 = 0;
    h->c1 = C;
    /* Step 1 initial state: Psi_t from the two-state profile (cell centres), Psi_p = 0 (reading). */
    for (int32_t i = 0; i < C; ++i) {
        double xc = p->x_min + ((double)i + 0.5) * h->c.dx;
        const ora_state *s = (xc < p->x_split) ? &p->left : &p->right;
        cons_of_state(s, p->R, h->psi + 5 * i);
        /* reading: the NTC majorant starts at 5 sqrt(2RT) of the initial cell state */
        h->cmax[i] = 5.0 * sqrt(2.0 * p->R * s->T);
    }
    return h;
}

void ora_destroy(void *vh)
{
    ora_inst *h = (ora_inst *)vh;
    if (!h) return;
    free(h->psi); free(h->avg); free(h->cmax); free(h->parts);
    free(h->ncand); free(h->nacc); free(h->nabs); free(h->nnew);
    free(h->last_flux); free(h->pre_m); free(h->post_m); free(h->F);
    free(h->lastpre); free(h->lastdest);
    free(h);
}

/* Free transport of one particle over dt in cell units, with the boundary conditions.
 * Returns the new cell in [0,C) or -1 if the particle left the domain.  The particle
 * position is cell-local, xl in [0,1).  Specular walls mirror the position (x -> 1 - x in
 * the mirrored cell) and the normal velocity, once per wall met. */
static int64_t transport(const ora_inst *h, int64_t cell, opart *q)
{
    const ora_params *p = &h->p;
    int64_t C = h->C;
    int64_t k;
    double xl;
    if (p->fp32) {
        float s = fmaf((float)q->u, h->c.dtdx_f, (float)q->xl);
        if (!(fabsf(s) < 1e15f)) return -1;   /* non-finite or absurd displacement: removed */
        float fk = floorf(s);
        float x = s - fk;
        k = (int64_t)fk;
        if (x >= 1.0f) { x = 0.0f; k += 1; }
        xl = (double)x;
    } else {
        double s = fma(q->u, h->c.dtdx, q->xl);
        if (!(fabs(s) < 1e15)) return -1;
        double fk = floor(s);
        double x = s - fk;
        k = (int64_t)fk;
        if (x >= 1.0) { x = 0.0; k += 1; }
        xl = x;
    }
    int64_t dest = cell + k;
    /* reading: a particle needing more than 64 wall reflections in one step is removed */
    for (int it = 0;; ++it) {
        if (it == 64) return -1;
        if (dest < 0) {
            if (p->bc_left == ORA_BC_SPECULAR) {
                dest = -dest - 1;
                xl = p->fp32 ? (double)(1.0f - (float)xl) : 1.0 - xl;
                if (xl >= 1.0) { xl = 0.0; dest += 1; }
                q->u = -q->u;
                continue;
            }
            if (p->bc_left == ORA_BC_PERIODIC) { dest = ((dest % C) + C) % C; continue; }
            return -1;
        }
        if (dest >= C) {
            if (p->bc_right == ORA_BC_SPECULAR) {
                dest = 2 * C - dest - 1;
                xl = p->fp32 ? (double)(1.0f - (float)xl) : 1.0 - xl;
                if (xl >= 1.0) { xl = 0.0; dest += 1; }
                q->u = -q->u;
                continue;
            }
            if (p->bc_right == ORA_BC_PERIODIC) { dest = dest % C; continue; }
            return -1;
        }
        break;
    }
    q->xl = xl;
    return dest;
}

/* exported for pin tests: transport one particle from `cell` and report the new cell */
int64_t ora_transport(void *vh, int64_t cell, double *xl, double *u)
{
    ora_inst *h = (ora_inst *)vh;
    opart q = { 0, *xl, *u, 0.0, 0.0 };
    int64_t d = transport(h, cell, &q);
    *xl = q.xl;
    *u = q.u;
    return d;
}

/* Collisions in one cell, NTC with VHS/HS (Appendix A).  `list` holds the N particles
 * of the cell after absorption and re-sampling; c_max persists per cell (reading). */
static void collide_cell(ora_inst *h, int32_t i, opart *list, int64_t N, double rho_t, int32_t *ncand,
                         int32_t *nacc)
{
    const ora_params *p = &h->p;
    const ora_consts *c = &h->c;
    *ncand = 0;
    *nacc = 0;
    if (N < 2) return;
    double rho_ratio;
    if (p->ntc_rate == ORA_NTC_TOTAL) rho_ratio = rho_t / p->rho_ref;
    else rho_ratio = ((double)N * c->mp / c->dx) / p->rho_ref;
    double cmax = h->cmax[i];
    double nsel = ntc_nsel(c, rho_ratio, (double)N, cmax);
    uint32_t w[4];
    draw(h->key, (uint32_t)(i + 1), 1u, h->step, ORA_ROUND, w);
    /* reading: stochastic rounding of the candidate count */
    double ncd = floor(nsel + ora_u53(w[0], w[1]));
    int64_t Nc = (int64_t)ncd;
    int32_t acc = 0;
    for (int64_t k = 0; k < Nc; ++k) {
        draw(h->key, (uint32_t)(i + 1), (uint32_t)(2 * k), h->step, ORA_COLLIDE, w);
        uint32_t a, b;
        ora_pick_pair(w[0], w[1], (uint32_t)N, &a, &b);
        opart *A = list + a, *B = list + b;
        double d0 = A->u - B->u, d1 = A->v - B->v, d2 = A->w - B->w;
        double cr = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        if (cr > cmax) cmax = cr;      /* reading: majorant raised before the test */
        double ua = ora_u53(w[2], w[3]);
        if (ua < accept_prob(c, cr, cmax)) {
            uint32_t v[4];
            draw(h->key, (uint32_t)(i + 1), (uint32_t)(2 * k + 1), h->step, ORA_COLLIDE, v);
            double va[3] = { A->u, A->v, A->w }, vb[3] = { B->u, B->v, B->w };
            ora_scatter(ora_u53(v[0], v[1]), ora_u53(v[2], v[3]), va, vb);
            A->u = st(p, va[0]); A->v = st(p, va[1]); A->w = st(p, va[2]);
            B->u = st(p, vb[0]); B->v = st(p, vb[1]); B->w = st(p, vb[2]);
            ++acc;
        }
    }
    h->cmax[i] = cmax;
    *ncand = (int32_t)Nc;
    *nacc = acc;
}

/* Number of particles re-sampled from the wave: stochastic rounding of
 * (1-P) max(rho_w, 0) dx / m_p (reading of "1-P of wave part converted"). */
static int64_t n_resample(const ora_inst *h, uint32_t id, double P, double rho_w)
{
    uint32_t w[4];
    draw(h->key, id, 0u, h->step, ORA_ROUND, w);
    double x = ((1.0 - P) * fmax(rho_w, 0.0)) * h->c.dx_over_mp;
    return (int64_t)floor(x + ora_u53(w[0], w[1]));
}

/* One step is taken in two halves, so that a domain split into parts (each part owning a range
 * of cells) can exchange the particles that cross into another part between them:
 *   first half  -- Step 1 (total state, split fraction, wave flux of the faces of the owned cells),
 *                  Step 2 of the owned cells (and of the inflow reservoirs at the domain's ends),
 *                  free transport of the resulting pre-transport array (Step 3);
 *   second half -- the owned cells' new particle lists (stable order by new cell; ties keep the
 *                  pre-transport order, which is cell-major over the whole domain), the particle
 *                  flux Eq. (fp), the conservative update Eq. (r1).
 * A whole-domain instance takes both halves in ora_step with nothing exchanged. */
static int step_first_half(ora_inst *h)
{
    const ora_params *p = &h->p;
    const ora_consts *c = &h->c;
    int32_t C = h->C;
    const int32_t c0 = h->c0, c1 = h->c1;
    ora_prim *W = (ora_prim *)malloc((size_t)C * sizeof(ora_prim));
    double *P = (double *)malloc((size_t)C * sizeof(double));
    double *F = h->F;
    int64_t *start = (int64_t *)malloc((size_t)(C + 1) * sizeof(int64_t));
    if (!W || !P || !start) { free(W); free(P); free(start); return -2; }
    {
        /* Step 1: total state and the split fraction of every cell */
        for (int32_t i = 0; i < C; ++i) {
            W[i] = prim_of_cons(h->psi + 5 * i, p->R);
            P[i] = pfrac(p, c, &W[i]);
        }
        /* wave flux at the faces of the owned cells from the start-of-step states */
        for (int32_t f = c0; f <= c1; ++f) {
            ora_prim L, Rr;
            if (f == 0) {
                Rr = W[0];
                if (p->bc_left == ORA_BC_PERIODIC) L = W[C - 1];
                else L = ghost_prim(h, 0, &W[0]);
            } else if (f == C) {
                L = W[C - 1];
                if (p->bc_right == ORA_BC_PERIODIC) Rr = W[0];
                else Rr = ghost_prim(h, 1, &W[C - 1]);
            } else {
                L = W[f - 1];
                Rr = W[f];
            }
            ora_prim LR = L, RR = Rr;
            if (p->recon_mode == ORA_RECON_VANLEER) {
                /* the states beyond L and R, and whether L and R are cells with a slope */
                const int per = (p->bc_left == ORA_BC_PERIODIC);
                ora_prim Wm, W2;
                memset(&Wm, 0, sizeof Wm);
                memset(&W2, 0, sizeof W2);
                int use0 = per || f - 1 >= 0, use1 = per || f < C;
                if (use0) {
                    int j = f - 2;
                    if (j >= 0) Wm = W[j];
                    else if (per) Wm = W[(j + C) % C];
                    else Wm = ghost_prim(h, 0, &W[0]);
                }
                if (use1) {
                    int j = f + 1;
                    if (j < C) W2 = W[j];
                    else if (per) W2 = W[j % C];
                    else W2 = ghost_prim(h, 1, &W[C - 1]);
                }
                recon_pair(&Wm, &L, &Rr, &W2, use0, use1, &LR, &RR);
            }
            wave_flux(p, c, &LR, &RR, &L, &Rr, 1, F + 5 * f);
        }
        if (p->bc_left == ORA_BC_PERIODIC && c0 == 0 && c1 == C) {
            /* the two boundary interfaces are the same interface */
            for (int k = 0; k < 5; ++k) F[5 * C + k] = F[k];
        }
        memcpy(h->last_flux + 5 * c0, F + 5 * c0, (size_t)(c1 - c0 + 1) * 5 * sizeof(double));

        /* cell starts in the sorted particle array (particles of the owned cells only) */
        for (int32_t i = 0; i <= C; ++i) start[i] = 0;
        for (int64_t q = 0; q < h->np; ++q) start[h->parts[q].cell + 1] += 1;
        for (int32_t i = 0; i < C; ++i) start[i + 1] += start[i];

        /* Step 2 per cell: absorb, re-sample, collide; build the pre-transport array,
         * ordered left ghost, cells 0..C-1, right ghost */
        opart *pre = NULL;
        int64_t npre = 0, cpre = 0;
        memset(h->pre_m, 0, (size_t)C * 5 * sizeof(double));
        /* left ghost reservoir (inflow boundary) */
        if (p->bc_left == ORA_BC_INOUT && c0 == 0) {
            ora_prim g = ghost_prim(h, 0, &W[0]);
            double Pg = pfrac(p, c, &g);
            int64_t ng = g.valid ? n_resample(h, 0u, Pg, g.rho) : 0;
            if (grow(h, &pre, &cpre, npre + ng)) return -2;
            for (int64_t j = 0; j < ng; ++j) {
                opart *q = pre + npre++;
                sample_particle(p, h->key, 0u, (uint32_t)j, h->step, &g, NULL, q);
                q->cell = -1;
            }
        }
        for (int32_t i = c0; i < c1; ++i) {
            int64_t n0 = start[i], n1 = start[i + 1];
            int64_t base = npre;
            if (grow(h, &pre, &cpre, npre + (n1 - n0))) return -2;
            int32_t nab = 0;
            for (int64_t k = n0; k < n1; ++k) {
                int absorbed = 0;
                if (P[i] > 0.0) {
                    uint32_t w[4];
                    draw(h->key, (uint32_t)(i + 1), (uint32_t)(k - n0), h->step, ORA_ABSORB, w);
                    absorbed = ora_u53(w[0], w[1]) < P[i];
                }
                if (absorbed) { ++nab; continue; }
                pre[npre++] = h->parts[k];
            }
            int64_t nsurv = npre - base;
            double rho_w = h->psi[5 * i] - (double)nsurv * c->mp_over_dx;
            int64_t nn = W[i].valid ? n_resample(h, (uint32_t)(i + 1), P[i], rho_w) : 0;
            if (grow(h, &pre, &cpre, npre + nn)) return -2;
            ora_ce ce;
            memset(&ce, 0, sizeof ce);
            if (p->resample_mode == ORA_RESAMPLE_CE && nn > 0) {
                /* neighbouring states as the wave flux sees them */
                ora_prim Wm, Wp;
                if (i > 0) Wm = W[i - 1];
                else if (p->bc_left == ORA_BC_PERIODIC) Wm = W[C - 1];
                else Wm = ghost_prim(h, 0, &W[0]);
                if (i < C - 1) Wp = W[i + 1];
                else if (p->bc_right == ORA_BC_PERIODIC) Wp = W[0];
                else Wp = ghost_prim(h, 1, &W[C - 1]);
                ce = ce_factor(p, c, &Wm, &W[i], &Wp);
            }
            for (int64_t j = 0; j < nn; ++j) {
                opart *q = pre + npre++;
                sample_particle(p, h->key, (uint32_t)(i + 1), (uint32_t)j, h->step, &W[i], &ce, q);
                q->cell = i;
            }
            collide_cell(h, i, pre + base, npre - base, h->psi[5 * i], &h->ncand[i], &h->nacc[i]);
            h->nabs[i] = nab;
            h->nnew[i] = (int32_t)nn;
            for (int64_t q = base; q < npre; ++q) add_phi(h->pre_m + 5 * i, pre + q);
        }
        if (p->bc_right == ORA_BC_INOUT && c1 == C) {
            ora_prim g = ghost_prim(h, 1, &W[C - 1]);
            double Pg = pfrac(p, c, &g);
            int64_t ng = g.valid ? n_resample(h, (uint32_t)(C + 1), Pg, g.rho) : 0;
            if (grow(h, &pre, &cpre, npre + ng)) return -2;
            for (int64_t j = 0; j < ng; ++j) {
                opart *q = pre + npre++;
                sample_particle(p, h->key, (uint32_t)(C + 1), (uint32_t)j, h->step, &g, NULL, q);
                q->cell = C;
            }
        }

        /* Step 3: free transport; particles leaving the domain are removed */
        int64_t *dest = (int64_t *)malloc((size_t)(npre ? npre : 1) * sizeof(int64_t));
        opart *moved = (opart *)malloc((size_t)(npre ? npre : 1) * sizeof(opart));
        if (!dest || !moved) { free(dest); free(moved); return -2; }
        int64_t nfar = 0;
        for (int64_t q = 0; q < npre; ++q) {
            moved[q] = pre[q];
            dest[q] = transport(h, pre[q].cell, &moved[q]);
            if (dest[q] >= 0) {
                int64_t d = dest[q] - pre[q].cell;
                if (d < -1 || d > 1) ++nfar;
            }
        }
        h->nfar = nfar;
        free(h->lastpre);
        free(h->lastdest);
        h->lastpre = pre;          /* kept: the pre-transport array of this step */
        h->lastdest = dest;
        h->nlastpre = npre;
        /* the transported records wait in .cell-less form for the second half */
        for (int64_t q = 0; q < npre; ++q) moved[q].cell = (int32_t)(dest[q] >= 0 ? dest[q] : -1);
        free(h->parts);
        h->parts = moved;
        h->cap = npre ? npre : 1;
        h->np = npre;
    }
    free(W); free(P); free(start);
    h->phase = 1;
    return 0;
}

/* The transported records of the first half whose new cell lies outside the owned range, in
 * pre-transport order (these go to the parts that own those cells). */
static int outside(const ora_inst *h, int64_t d) { return d >= 0 && (d < h->c0 || d >= h->c1); }

int64_t ora_outbox_count(void *vh)
{
    ora_inst *h = (ora_inst *)vh;
    int64_t n = 0;
    if (h->phase != 1) return -1;
    for (int64_t q = 0; q < h->np; ++q) n += outside(h, h->parts[q].cell);
    return n;
}

void ora_outbox(void *vh, int32_t *cell, double *xl, double *u, double *v, double *w)
{
    ora_inst *h = (ora_inst *)vh;
    int64_t n = 0;
    for (int64_t q = 0; q < h->np; ++q) {
        const opart *r = h->parts + q;
        if (!outside(h, r->cell)) continue;
        cell[n] = r->cell; xl[n] = r->xl; u[n] = r->u; v[n] = r->v; w[n] = r->w;
        ++n;
    }
}

/* Second half.  lo / hi: the transported records arriving from parts that own lower / higher cells,
 * each in the pre-transport order of the whole domain (by source part, then that part's order).
 * The new list of an owned cell is then [from lower parts] [from this part] [from higher parts],
 * each in pre-transport order -- the stable order by new cell of the undivided array. */
static int step_second_half(ora_inst *h, int64_t nlo, const opart *lo, int64_t nhi, const opart *hi)
{
    const ora_params *p = &h->p;
    const ora_consts *c = &h->c;
    int32_t C = h->C;
    const int32_t c0 = h->c0, c1 = h->c1;
    if (h->phase != 1) return -1;
    const double *F = h->F;
    opart *mv = h->parts;
    int64_t nmv = h->np;
    /* stable counting sort by the new cell over lo ++ own ++ hi */
    int64_t *cnt = (int64_t *)calloc((size_t)C + 1, sizeof(int64_t));
    if (!cnt) return -2;
    for (int64_t q = 0; q < nlo; ++q) {
        if (lo[q].cell < c0 || lo[q].cell >= c1) { free(cnt); return -1; }
        cnt[lo[q].cell + 1] += 1;
    }
    for (int64_t q = 0; q < nmv; ++q)
        if (mv[q].cell >= c0 && mv[q].cell < c1) cnt[mv[q].cell + 1] += 1;
    for (int64_t q = 0; q < nhi; ++q) {
        if (hi[q].cell < c0 || hi[q].cell >= c1) { free(cnt); return -1; }
        cnt[hi[q].cell + 1] += 1;
    }
    for (int32_t i = 0; i < C; ++i) cnt[i + 1] += cnt[i];
    int64_t nkeep = cnt[C];
    opart *np_ = (opart *)malloc((size_t)(nkeep ? nkeep : 1) * sizeof(opart));
    if (!np_) { free(cnt); return -2; }
    for (int64_t q = 0; q < nlo; ++q) np_[cnt[lo[q].cell]++] = lo[q];
    for (int64_t q = 0; q < nmv; ++q)
        if (mv[q].cell >= c0 && mv[q].cell < c1) np_[cnt[mv[q].cell]++] = mv[q];
    for (int64_t q = 0; q < nhi; ++q) np_[cnt[hi[q].cell]++] = hi[q];
    free(cnt);
    free(h->parts);
    h->parts = np_;
    h->cap = nkeep ? nkeep : 1;
    h->np = nkeep;

    /* particle flux Eq. (fp) = change of the per-cell particle moments over the
     * transport; wave flux by the NS solver; conservative update Eq. (r1) */
    memset(h->post_m, 0, (size_t)C * 5 * sizeof(double));
    for (int64_t q = 0; q < h->np; ++q) add_phi(h->post_m + 5 * h->parts[q].cell, h->parts + q);
    for (int32_t i = c0; i < c1; ++i) {
        for (int k = 0; k < 5; ++k) {
            double fp = c->mp_over_dx * (h->post_m[5 * i + k] - h->pre_m[5 * i + k]);
            double fw = c->dtdx * (F[5 * (i + 1) + k] - F[5 * i + k]);
            h->psi[5 * i + k] = h->psi[5 * i + k] + fp - fw;
        }
    }
    h->step += 1;
    if ((int64_t)h->step > (int64_t)p->avg_start) {
        for (int64_t k = (int64_t)c0 * 5; k < (int64_t)c1 * 5; ++k) h->avg[k] += h->psi[k];
        h->navg += 1;
    }
    h->phase = 0;
    return 0;
}

int ora_step(void *vh, int32_t nsteps)
{
    ora_inst *h = (ora_inst *)vh;
    if (h->c0 != 0 || h->c1 != h->C || h->phase != 0) return -1;
    for (int32_t s = 0; s < nsteps; ++s) {
        int rc = step_first_half(h);
        if (rc) return rc;
        rc = step_second_half(h, 0, NULL, 0, NULL);
        if (rc) return rc;
    }
    return 0;
}

/* Domain decomposition (host-rank emulation): this instance owns cells [c0, c1) of the domain.
 * Set before the first step, on an instance without particles.  The states of the cells next to
 * the owned range (two on each side, periodic ends wrapping) must be set by the caller before
 * every first half (ora_set_psi) from the parts that own them. */
int ora_set_range(void *vh, int32_t c0, int32_t c1)
{
    ora_inst *h = (ora_inst *)vh;
    if (c0 < 0 || c1 > h->C || c0 >= c1 || h->np != 0 || h->phase != 0) return -1;
    h->c0 = c0;
    h->c1 = c1;
    return 0;
}

int ora_step_first_half(void *vh)
{
    ora_inst *h = (ora_inst *)vh;
    if (h->phase != 0) return -1;
    return step_first_half(h);
}

int ora_step_second_half(void *vh, int64_t nlo, const int32_t *lc, const double *lxl, const double *lu,
                         const double *lv, const double *lw, int64_t nhi, const int32_t *hc, const double *hxl,
                         const double *hu, const double *hv, const double *hw)
{
    ora_inst *h = (ora_inst *)vh;
    opart *lo = (opart *)malloc((size_t)(nlo ? nlo : 1) * sizeof(opart));
    opart *hi = (opart *)malloc((size_t)(nhi ? nhi : 1) * sizeof(opart));
    if (!lo || !hi) { free(lo); free(hi); return -2; }
    for (int64_t q = 0; q < nlo; ++q) { lo[q].cell = lc[q]; lo[q].xl = lxl[q]; lo[q].u = lu[q]; lo[q].v = lv[q]; lo[q].w = lw[q]; }
    for (int64_t q = 0; q < nhi; ++q) { hi[q].cell = hc[q]; hi[q].xl = hxl[q]; hi[q].u = hu[q]; hi[q].v = hv[q]; hi[q].w = hw[q]; }
    int rc = step_second_half(h, nlo, lo, nhi, hi);
    free(lo);
    free(hi);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Accessors                                                                   */
/* ------------------------------------------------------------------------- */
int64_t ora_num_particles(void *vh) { return ((ora_inst *)vh)->np; }
int64_t ora_num_last_pre(void *vh) { return ((ora_inst *)vh)->nlastpre; }

/* the last step's pre-transport array: source cell (-1 / C for the ghost reservoirs),
 * destination cell (-1: removed), and the record before transport */
void ora_get_last_pre(void *vh, int32_t *src, int64_t *dest, double *xl, double *u, double *v, double *w)
{
    ora_inst *h = (ora_inst *)vh;
    for (int64_t q = 0; q < h->nlastpre; ++q) {
        src[q] = h->lastpre[q].cell;
        dest[q] = h->lastdest[q];
        xl[q] = h->lastpre[q].xl;
        u[q] = h->lastpre[q].u;
        v[q] = h->lastpre[q].v;
        w[q] = h->lastpre[q].w;
    }
}
uint32_t ora_step_count(void *vh) { return ((ora_inst *)vh)->step; }
int64_t ora_last_nfar(void *vh) { return ((ora_inst *)vh)->nfar; }

void ora_get_particles(void *vh, int32_t *cell, double *xl, double *u, double *v, double *w)
{
    ora_inst *h = (ora_inst *)vh;
    for (int64_t q = 0; q < h->np; ++q) {
        cell[q] = h->parts[q].cell;
        xl[q] = h->parts[q].xl;
        u[q] = h->parts[q].u;
        v[q] = h->parts[q].v;
        w[q] = h->parts[q].w;
    }
}

/* Replace the particle set (test hook: e.g. an anisotropic start for relaxation tests).
 * The arrays must be sorted by cell. */
int ora_set_particles(void *vh, int64_t n, const int32_t *cell, const double *xl, const double *u,
                      const double *v, const double *w)
{
    ora_inst *h = (ora_inst *)vh;
    if (n > h->cap) {
        opart *na = (opart *)realloc(h->parts, (size_t)(n ? n : 1) * sizeof(opart));
        if (!na) return -2;
        h->parts = na;
        h->cap = n;
    }
    for (int64_t q = 0; q < n; ++q) {
        if (cell[q] < 0 || cell[q] >= h->C) return -1;
        if (q > 0 && cell[q] < cell[q - 1]) return -1;
        h->parts[q].cell = cell[q];
        h->parts[q].xl = st(&h->p, xl[q]);
        h->parts[q].u = st(&h->p, u[q]);
        h->parts[q].v = st(&h->p, v[q]);
        h->parts[q].w = st(&h->p, w[q]);
    }
    h->np = n;
    return 0;
}

void ora_get_psi(void *vh, double *out) { ora_inst *h = (ora_inst *)vh; memcpy(out, h->psi, (size_t)h->C * 5 * sizeof(double)); }
void ora_set_psi(void *vh, const double *in) { ora_inst *h = (ora_inst *)vh; memcpy(h->psi, in, (size_t)h->C * 5 * sizeof(double)); }
int64_t ora_get_avg(void *vh, double *out) { ora_inst *h = (ora_inst *)vh; memcpy(out, h->avg, (size_t)h->C * 5 * sizeof(double)); return h->navg; }
void ora_get_cmax(void *vh, double *out) { ora_inst *h = (ora_inst *)vh; memcpy(out, h->cmax, (size_t)h->C * sizeof(double)); }
void ora_get_last_flux(void *vh, double *out) { ora_inst *h = (ora_inst *)vh; memcpy(out, h->last_flux, (size_t)(h->C + 1) * 5 * sizeof(double)); }
void ora_get_last_moments(void *vh, double *pre, double *post)
{
    ora_inst *h = (ora_inst *)vh;
    memcpy(pre, h->pre_m, (size_t)h->C * 5 * sizeof(double));
    memcpy(post, h->post_m, (size_t)h->C * 5 * sizeof(double));
}

void ora_get_counters(void *vh, int32_t *ncand, int32_t *nacc, int32_t *nabs, int32_t *nnew)
{
    ora_inst *h = (ora_inst *)vh;
    memcpy(ncand, h->ncand, (size_t)h->C * sizeof(int32_t));
    memcpy(nacc, h->nacc, (size_t)h->C * sizeof(int32_t));
    memcpy(nabs, h->nabs, (size_t)h->C * sizeof(int32_t));
    memcpy(nnew, h->nnew, (size_t)h->C * sizeof(int32_t));
}

/* derived constants: dx, dt, dtdx, mp, beta, lambda_ref, mu_ref, upsilon, c_ref, ntc_A */
void ora_get_consts(void *vh, double out[10])
{
    ora_inst *h = (ora_inst *)vh;
    const ora_consts *c = &h->c;
    out[0] = c->dx; out[1] = c->dt; out[2] = c->dtdx; out[3] = c->mp; out[4] = c->beta;
    out[5] = c->lambda_ref; out[6] = c->mu_ref; out[7] = c->upsilon; out[8] = c->c_ref; out[9] = c->ntc_A;
}

/* Normal stress Pi = S_xx and heat flux Q = Q_x of every cell (Eq. gkt_moment1: S is the second
 * central moment of f - g, Q the third of f) from the current state.  The distribution is the
 * particles plus the wave (Step 1):
 *   particles: central moments about the total velocity U_t of the cell,
 *     S_p = (m_p/dx) sum (xi_x - U)^2 - rho_p R T_t,  Q_p = (m_p/dx) sum (xi_x - U) |xi - U|^2 / 2,
 *     rho_p = n m_p / dx (the Maxwellian g at the total state takes rho_t R T_t; the wave's
 *     Maxwellian part takes rho_w R T_t of it back, leaving rho_p R T_t);
 *   wave (reading): its NS stress and heat flux, the values the Chapman-Enskog re-sampling uses
 *     (neighbour states as the wave flux sees them, mu_e = eps mu), weighted by rho_w / rho_t.
 * A cell whose total state is not usable (rho_t <= 0 or T_t <= 0) reports 0 for both. */
void ora_stress_heat(void *vh, double *Pi, double *Q)
{
    ora_inst *h = (ora_inst *)vh;
    const ora_params *p = &h->p;
    const ora_consts *c = &h->c;
    const int32_t C = h->C;
    ora_prim *W = (ora_prim *)malloc((size_t)C * sizeof(ora_prim));
    double *s2 = (double *)calloc((size_t)C, sizeof(double));
    double *s3 = (double *)calloc((size_t)C, sizeof(double));
    int64_t *n = (int64_t *)calloc((size_t)C, sizeof(int64_t));
    if (!W || !s2 || !s3 || !n) {
        free(W); free(s2); free(s3); free(n);
        for (int32_t i = 0; i < C; ++i) Pi[i] = Q[i] = NAN;
        return;
    }
    for (int32_t i = 0; i < C; ++i) W[i] = prim_of_cons(h->psi + 5 * i, p->R);
    for (int64_t k = 0; k < h->np; ++k) {
        const opart *q = h->parts + k;
        const int32_t i = q->cell;
        const double cx = q->u - W[i].u, cy = q->v - W[i].v, cz = q->w - W[i].w;
        s2[i] += cx * cx;
        s3[i] += cx * (0.5 * (cx * cx + cy * cy + cz * cz));
        n[i] += 1;
    }
    for (int32_t i = 0; i < C; ++i) {
        Pi[i] = Q[i] = 0.0;
        if (!W[i].valid) continue;
        const double rho_p = (double)n[i] * c->mp_over_dx;
        Pi[i] = c->mp_over_dx * s2[i] - rho_p * p->R * W[i].T;
        Q[i] = c->mp_over_dx * s3[i];
        ora_prim Wm, Wp;
        if (i > 0) Wm = W[i - 1];
        else if (p->bc_left == ORA_BC_PERIODIC) Wm = W[C - 1];
        else Wm = ghost_prim(h, 0, &W[0]);
        if (i < C - 1) Wp = W[i + 1];
        else if (p->bc_right == ORA_BC_PERIODIC) Wp = W[0];
        else Wp = ghost_prim(h, 1, &W[C - 1]);
        const ora_ce f = ce_factor(p, c, &Wm, &W[i], &Wp);
        const double rho_t = h->psi[5 * i];
        const double wgt = (rho_t - rho_p) / rho_t;
        Pi[i] += wgt * f.sxx;
        Q[i] += wgt * f.qx;
    }
    free(W); free(s2); free(s3); free(n);
}

/* primitive state and P of every cell from the current Psi_t */
void ora_get_prim(void *vh, double *rho, double *u, double *T, double *P, int32_t *valid)
{
    ora_inst *h = (ora_inst *)vh;
    for (int32_t i = 0; i < h->C; ++i) {
        ora_prim q = prim_of_cons(h->psi + 5 * i, h->p.R);
        rho[i] = q.rho; u[i] = q.u; T[i] = q.T; valid[i] = q.valid;
        P[i] = pfrac(&h->p, &h->c, &q);
    }
}

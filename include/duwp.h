/*
 * duwp.h -- C ABI of the GB300 (sm_103a) library for the per-time-step hot path of the
 * direct unified wave-particle (DUWP) method (Cao, Liu, Yang, Zhong, arXiv 2305.12071).
 *
 * One time step of one instance (Sec. 3.4, "Algorithm of DUWP", Steps 1-4):
 *   - total state Psi_t = Psi_w + Psi_p per cell (Step 1);
 *   - P of the particles of a cell absorbed into the wave, P from Eq. (p); (1-P) of the
 *     wave re-sampled as Maxwellian particles at the total state, Eq. (maxsample);
 *     NTC pair selection with VHS collisions on the particle part (Step 2, Appendix A);
 *   - free transport x += xi dt with boundary handling, the particle flux of Eq. (fp),
 *     an NS wave flux with the viscosity correction eps of Eq. (vp1), and the
 *     conservative update of Eq. (r1) (Step 3).
 * The problem is posed as in Sec. 4: gas and VHS constants, mesh, Knudsen number,
 * time step and boundary states.
 *
 * Conventions for every function below:
 *   - return value: DUWP_OK (0) or a negative DUWP_E* status; DUWP_PENDING (1) only
 *     from duwp_poll;
 *   - pointers named host_* or documented as host buffers are caller-owned host memory;
 *     the library owns all device memory it allocates (through the caller's allocator
 *     callbacks when given, cudaMallocAsync on the handle's stream otherwise);
 *   - a handle is not thread-safe; a server is safe for concurrent submit/poll;
 *   - work is enqueued on the CUDA stream given at creation; functions documented as
 *     "synchronizing" wait for that stream and report any error recorded on the device
 *     (a cell or buffer overflow inside a step) as their status.  After a failed step
 *     the handle may only be destroyed.
 */
#ifndef DUWP_H
#define DUWP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
enum {
    DUWP_OK = 0,
    DUWP_EINVAL = -1,     /* invalid argument or problem description */
    DUWP_ENOMEM = -2,     /* an allocation failed (host or device) */
    DUWP_ECUDA = -3,      /* a CUDA call failed; see duwp_last_cuda_error() */
    DUWP_ENUMERIC = -4,   /* non-finite or non-physical state uploaded or produced */
    DUWP_ETIMEOUT = -5,   /* a bounded device wait ran out */
    DUWP_EBUSY = -6,      /* server: request cannot be admitted now / queue full */
    DUWP_EOVERFLOW = -7,  /* a cell, the particle buffers or the far-mover list overflowed */
    DUWP_ENOTFOUND = -8,  /* server: unknown request id */
    DUWP_PENDING = 1      /* server: request not finished yet */
};

/* ------------------------------------------------------------------ problem description */
/* A macroscopic state (density, velocity components, temperature). */
typedef struct { double rho, u, v, w, T; } duwp_state;

enum {
    DUWP_BC_INOUT = 0,     /* reservoir at the fixed boundary state: particles leaving are removed,
                              inflow particles are sampled each step from the boundary state */
    DUWP_BC_SPECULAR = 1,  /* specular wall: x and the normal velocity are mirrored */
    DUWP_BC_PERIODIC = 2,  /* periodic (both ends must be periodic) */
    DUWP_BC_VACUUM = 3     /* outflow into vacuum: particles leaving are removed, nothing enters */
};
enum { DUWP_FP64 = 0, DUWP_FP32 = 1 };                       /* particle record precision */
enum { DUWP_EPS1 = 0, DUWP_EPS12 = 1, DUWP_EPS0 = 2, DUWP_EPS_AVG = 3 }; /* Sec. 3.3 */
enum { DUWP_FLUX_GKS_EQ = 0, DUWP_FLUX_KFVS = 1 };           /* wave-flux form */
enum { DUWP_NTC_PARTICLE = 0, DUWP_NTC_TOTAL = 1 };          /* density in the NTC count */
enum { DUWP_RESAMPLE_MAXWELL = 0, DUWP_RESAMPLE_CE = 1 };    /* velocity law of re-sampled particles */
enum { DUWP_SPLIT_P = 0, DUWP_SPLIT_QMC = 1 };              /* wave/particle split fraction */
enum { DUWP_RECON_FIRST = 0, DUWP_RECON_VANLEER = 1 };       /* wave-flux interface states */

/*
 * Problem parameters of one instance (Sec. 4 and Appendix A; units nondimensional):
 *   gamma, Pr, R        gas constants (5/3, 2/3, 1 for argon);
 *   omega, alpha        VHS viscosity index and the alpha of beta in Eq. (lambda);
 *   rho_ref, T_ref      reference state; Kn * L_ref is the reference mean free path,
 *                       which fixes mu_ref through Eq. (lambda) (first form);
 *   x_min, x_max, n_cells   uniform 1D mesh;
 *   dt                  time step; if dt <= 0 it is cfl * dx / max(|u| + 3 sqrt(2 R T)) over
 *                       the two initial states;
 *   left, right, x_split   initial states left/right of x_split (cell centres decide);
 *                       they are also the reservoir states of DUWP_BC_INOUT ends;
 *   bc_left, bc_right   boundary kinds (DUWP_BC_*);
 *   ppc_ref             simulated particles per cell at rho_ref: m_p = rho_ref dx / ppc_ref;
 *   precision           DUWP_FP64 or DUWP_FP32 particle records (all cell quantities are FP64);
 *   eps_mode, flux_mode, ntc_rate   options (DUWP_EPS*, DUWP_FLUX_*, DUWP_NTC_*);
 *   seed                key of the counter-based generator of this instance;
 *   capacity            particle slots per buffer (0: automatic; each cell's output block takes
 *                       twice the bound on its list after re-sampling);
 *   avg_start           time averages accumulate the states after step avg_start;
 *   resample_mode       velocities of the particles drawn from the wave (Sec. 3.4, Step 2):
 *                       DUWP_RESAMPLE_MAXWELL (default, Eq. maxsample: the local Maxwellian) or
 *                       DUWP_RESAMPLE_CE (the local Maxwellian times its first-order
 *                       Chapman-Enskog factor, Eq. ce2, with the NS stress and heat flux of the
 *                       wave from central differences of the neighbouring cells and the viscosity
 *                       eps mu of the flux; drawn by acceptance-rejection against 1 + 30 B, B the
 *                       largest normalised stress or heat flux; Maxwellian where B > 1/4 and in the
 *                       inflow reservoirs);
 *   split_mode          the split fraction of Step 2 and the weight of the wave flux (Step 3):
 *                       DUWP_SPLIT_P (default, Eq. p: P = max(0, 1 - tau/dt), the flux weighted by
 *                       max(0, 1 - tau_f/dt)) or DUWP_SPLIT_QMC (the multi-scale Boltzmann
 *                       equation's quantified model competition, Sec. 3.2: particles collide --
 *                       are absorbed into the wave -- with probability 1 - exp(-dt/tau), and the
 *                       flux of Sec. 3.3 at t = dt is weighted by 1 - exp(-dt/tau_f));
 *   recon_mode          interface states of the wave flux: DUWP_RECON_FIRST (default, the two
 *                       cell states) or DUWP_RECON_VANLEER (second order: per primitive variable
 *                       the van Leer limited slope 2 dl dr / (dl + dr) of each cell, zero at
 *                       extrema and in reservoir / mirror cells, the interface seeing each cell's
 *                       state plus or minus half its slope; the NS gradients still from the cell
 *                       states).
 * In a batch all instances must use the same precision.
 */
typedef struct {
    double gamma, Pr, R;
    double omega, alpha;
    double rho_ref, T_ref, Kn, L_ref;
    double x_min, x_max;
    int32_t n_cells;
    double dt, cfl;
    duwp_state left, right;
    double x_split;
    int32_t bc_left, bc_right;
    double ppc_ref;
    int32_t precision, eps_mode, flux_mode, ntc_rate;
    uint64_t seed;
    uint64_t capacity;
    int32_t avg_start;
    int32_t resample_mode;
    int32_t split_mode;
    int32_t recon_mode;
} duwp_params;

/* Device allocator callbacks: alloc returns device memory of `bytes` bytes usable on `stream`
 * (NULL on failure); free releases it.  `ctx` is passed through unchanged. */
typedef void *(*duwp_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*duwp_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

typedef struct duwp_handle duwp_handle;

/* Derived constants of one instance (Sec. 4.1 Eq. lambda, Appendix A). */
typedef struct {
    double dx, dt, mp, beta, lambda_ref, mu_ref, c_ref;
    int64_t capacity;        /* particle slots per buffer of the whole handle */
    int32_t n_instances;
    int64_t steps_done;      /* steps taken by this instance */
    int64_t particle_updates;/* particles streamed through a step by this instance, all steps so far */
} duwp_info;

/* ------------------------------------------------------------------ single instance and batch */

/* Create one DUWP instance on the CUDA `stream` (cudaStream_t, NULL = legacy default).
 * The initial state is all wave: Psi_t from the two-state profile and no particles; the
 * first step samples the particle part (Step 1 of Sec. 3.4).  Allocates through
 * alloc/free_fn when both are non-NULL.  Errors: DUWP_EINVAL (bad parameters), DUWP_ENOMEM,
 * DUWP_ECUDA.  On success *out owns the device state until duwp_destroy. */
int duwp_init(const duwp_params *params, void *stream, duwp_alloc_fn alloc, duwp_free_fn free_fn,
              void *alloc_ctx, duwp_handle **out);

/* Create `n` independent instances stepped together by one set of launches over a flattened
 * cell index (batched form; instances never exchange data).  params[i] describes instance i;
 * all share one precision.  Same errors and ownership as duwp_init. */
int duwp_init_batch(const duwp_params *params, int32_t n, void *stream, duwp_alloc_fn alloc,
                    duwp_free_fn free_fn, void *alloc_ctx, duwp_handle **out);

/* Advance every instance of the handle by n_steps >= 0 DUWP steps (Steps 1-4 of Sec. 3.4).
 * Asynchronous on the handle's stream: device-side overflows are reported by the next
 * synchronizing call.  Errors: DUWP_EINVAL, DUWP_ECUDA. */
int duwp_step(duwp_handle *h, int32_t n_steps);

/* Synchronizing: wait for the handle's stream; returns the device error status. */
int duwp_sync(duwp_handle *h);

/* Synchronizing.  Advance by n_steps >= 1 steps as individual launches with CUDA events recorded
 * on the handle's stream around every kernel.  host_kernel_ms[DUWP_TIMED_SLOTS] (caller-owned)
 * receives the summed device time of [0] the collision kernel (collisions of the cells with
 * P = 0 and the re-sampled particles of the cells without collisions), [1] the streaming kernel
 * (transport and sorted runs of every particle), [2] the far-mover sort, [3] the cell update,
 * [4] the offset kernel and the wave-flux kernel (run at the start of the step that applies the
 * flux, beside the particle kernels in duwp_step) and [6] the kernels ahead of the collision kernel (the
 * re-sampled particles of cells with many of them, then absorption, re-sampling and collisions of
 * the cells with many collision candidates), and in [5] the device time from the first launch to
 * the end of the last; host_step_ms (n_steps entries, may be NULL) the device time of each step.
 * Results are identical to duwp_step.  Errors: as duwp_step and duwp_sync. */
enum { DUWP_TIMED_SLOTS = 7 };
int duwp_step_timed(duwp_handle *h, int32_t n_steps, double *host_kernel_ms, double *host_step_ms);

enum { DUWP_INSTANT = 0, DUWP_AVERAGED = 1 };

/* Synchronizing.  Macroscopic profile of instance `inst` into caller-owned HOST arrays of
 * n = n_cells doubles: density, x-velocity and temperature of the total state Psi_t
 * (which = DUWP_INSTANT) or of its time average (DUWP_AVERAGED, over the states after step
 * avg_start), and the wave fraction rho_w / rho_t of the current state (Fig. 5f).  Any of the
 * output pointers may be NULL.  Errors: DUWP_EINVAL (inst or n), device errors. */
int duwp_moments(duwp_handle *h, int32_t inst, int32_t which, double *host_rho, double *host_u,
                 double *host_T, double *host_wave_frac, int32_t n);

/* Synchronizing.  duwp_moments for every active instance of the handle at once: one device pass
 * and one copy per output array.  The caller-owned HOST arrays hold total_cells doubles each (the
 * sum of n_cells over the active instances); instance b's cells follow those of the active
 * instances with smaller index.  Any of the output pointers may be NULL.  The values are those of
 * duwp_moments bit for bit.  Errors: DUWP_EINVAL (which, or total_cells not the sum), DUWP_ENOMEM
 * (its device scratch, 64 B per cell, kept by the handle), device errors. */
int duwp_moments_all(duwp_handle *h, int32_t which, double *host_rho, double *host_u, double *host_T,
                     double *host_wave_frac, int64_t total_cells);

/* Non-blocking.  duwp_moments_all of the state reached by the steps enqueued so far: the profile
 * pass is enqueued behind them and the copies into the caller's HOST arrays run on a separate
 * stream, so the caller may enqueue the next steps at once and they overlap with the copies (the
 * arrays must be pinned for that; with pageable arrays the call blocks until its copies are done).
 * The arrays (same layout as duwp_moments_all) must stay valid, and are not to be read, until
 * duwp_moments_wait (or any synchronizing call) returns.  Reads complete in call order; at most two
 * are in flight (a third waits on the device, not the host, for the first one's copies).  Values
 * equal those of duwp_moments_all bit for bit.  Errors: DUWP_EINVAL (which, or total_cells not the
 * sum), DUWP_ENOMEM (scratch, 64 B per cell); device errors are reported by the next synchronizing
 * call. */
int duwp_moments_all_async(duwp_handle *h, int32_t which, double *host_rho, double *host_u, double *host_T,
                           double *host_wave_frac, int64_t total_cells);

/* Blocks until every read enqueued by duwp_moments_all_async has landed in its host arrays (the steps
 * enqueued after them may still run).  Errors: DUWP_EINVAL (h), device errors. */
int duwp_moments_wait(duwp_handle *h);

/* Synchronizing.  Conservative total state Psi_t = (rho, rho U, rho V, rho W, rho E) per cell of
 * instance `inst` (which = DUWP_INSTANT) or its time average (DUWP_AVERAGED) into a caller-owned
 * host array of n_cells * 5 doubles, cell-major.  *host_navg (may be NULL) receives the number of
 * averaged states. */
int duwp_fields(duwp_handle *h, int32_t inst, int32_t which, double *host_psi, int32_t n_cells,
                int64_t *host_navg);

/* Synchronizing.  Normal stress Pi = S_xx and heat flux Q = Q_x (Sec. 2, Eq. gkt_moment1: S the
 * second central moment of f - g, Q the third of f) per cell of instance `inst` into caller-owned
 * HOST arrays of n = n_cells doubles.  f is the particles plus the wave: the particle part from the
 * central moments of the cell's particles about the total velocity U_t,
 *   (m_p/dx) sum (xi_x - U)^2 - rho_p R T_t   and   (m_p/dx) sum (xi_x - U) |xi - U|^2 / 2,
 * the wave part its Navier-Stokes stress -(4/3) mu_e dU/dx and heat flux -(5/2) R mu_e / Pr dT/dx
 * (mu_e = eps mu at the cell's state, central differences over the neighbouring states as the wave
 * flux sees them) weighted by rho_w / rho_t.  A cell whose total state is not usable reports 0.
 * which = DUWP_INSTANT: of the current state (one device pass over the instance's particles);
 * DUWP_AVERAGED: the mean of the values taken by duwp_stress_heat_accumulate so far (0 before the
 * first).  Errors: DUWP_EINVAL (inst, which, n, NULL arrays), DUWP_ENOMEM (its device scratch,
 * 72 B per cell, kept by the handle), device errors. */
int duwp_stress_heat(duwp_handle *h, int32_t inst, int32_t which, double *host_Pi, double *host_Q, int32_t n);

/* Non-blocking.  Adds the current Pi and Q of every cell of every instance (as duwp_stress_heat
 * DUWP_INSTANT computes them) to the handle's running sums: enqueued behind the steps enqueued so
 * far, one call per state to be averaged (for the time-averaged profiles of Sec. 4.1, after each
 * step from the first averaged one).  The sums are not part of a checkpoint.  Errors: DUWP_EINVAL
 * (h), DUWP_ENOMEM (scratch); device errors are reported by the next synchronizing call. */
int duwp_stress_heat_accumulate(duwp_handle *h);

/* Shock-structure profiles in the paper's normalisation (Sec. 4.1; host arithmetic, no device
 * work).  From n values per cell of position x, density, temperature, normal stress Pi and heat flux
 * Q (caller-owned host arrays; the outputs may alias the inputs), with the inflow state
 * (rho_up, T_up), the outflow state (rho_down, T_down), the inflow mean free path lam_up of
 * Eq. (lambda) and its factor beta, and the gas constant R:
 *   DUWP_SHOCK_MA3 (Eq. ma3): rho/rho_up, T/T_up, Pi/p_up, Q/(p_up sqrt(2 R T_up)), x/(sqrt(pi) lam_up/2);
 *   DUWP_SHOCK_MA8 (Eq. ma8): (rho - rho_up)/(rho_down - rho_up), (T - T_up)/(T_down - T_up),
 *                             Pi/(rho_up 2 R T_up), Q/(rho_up (2 R T_up)^(3/2)), x/(beta pi lam_up);
 * p_up = rho_up R T_up.  Any output pointer may be NULL.  Errors: DUWP_EINVAL (kind, n < 0, NULL
 * inputs for a requested output, non-positive scales). */
enum { DUWP_SHOCK_MA3 = 0, DUWP_SHOCK_MA8 = 1 };
int duwp_shock_normalise(int32_t kind, int64_t n, const double *x, const double *rho, const double *T,
                         const double *Pi, const double *Q, double rho_up, double T_up, double rho_down,
                         double T_down, double lam_up, double beta, double R, double *x_out, double *rho_out,
                         double *T_out, double *Pi_out, double *Q_out);

/* Derived constants and sizes of instance `inst` (not synchronizing except steps_done). */
int duwp_get_info(duwp_handle *h, int32_t inst, duwp_info *out);

/* Release every device allocation of the handle (after waiting for its stream). */
int duwp_destroy(duwp_handle *h);

/* Static description of a status code. */
const char *duwp_error_string(int status);

/* Text of the last CUDA error seen by this library in the calling thread (static storage). */
const char *duwp_last_cuda_error(void);

/* ------------------------------------------------------------------ launch configuration */

/* Launch shape of the streaming kernel (one warp per cell): threads per block (multiple of 32,
 * 32..512), the register budget (reg_capped = 0: up to 128 registers per thread; 1: up to 64,
 * two 512-thread blocks per SM; 2: up to 40, three) and the particles each thread has in flight
 * (groups = 2 or 3 groups of 32 records per warp loaded before any is processed).  Used by the
 * autotuner; results do not depend on it.
 * Synchronizing.  Errors: DUWP_EINVAL for shapes the device cannot launch. */
int duwp_set_launch(duwp_handle *h, int32_t threads, int32_t reg_capped, int32_t groups);

/* Capture the per-step launches in CUDA graphs (on = 1, default) or launch them one by one
 * (on = 0, the plain loop). */
int duwp_use_graphs(duwp_handle *h, int32_t on);

/* ------------------------------------------------------------------ inspection (tests, checkpoints) */

/* Synchronizing.  Number of particles of instance `inst` (all cells). */
int duwp_num_particles(duwp_handle *h, int32_t inst, int64_t *out);

/* Synchronizing.  Particles of instance `inst` in the stable per-cell order the method defines
 * (sorted by cell; within a cell by their order before the last transport), into caller-owned
 * host arrays of n entries (n = duwp_num_particles): cell index, cell-local position in [0,1),
 * velocity.  Errors: DUWP_EINVAL if n differs. */
int duwp_get_particles(duwp_handle *h, int32_t inst, int32_t *host_cell, double *host_xl,
                       double *host_u, double *host_v, double *host_w, int64_t n);

/* Synchronizing.  Per-cell counters of the last step of instance `inst` (host arrays of n_cells
 * int32, any may be NULL): NTC candidates, accepted collisions, absorbed particles, re-sampled
 * particles. */
int duwp_get_counters(duwp_handle *h, int32_t inst, int32_t *host_ncand, int32_t *host_nacc,
                      int32_t *host_nabs, int32_t *host_nnew, int32_t n_cells);

/* Synchronizing.  Per-cell NTC majorant c_r,max of instance `inst` (host, n_cells doubles). */
int duwp_get_cmax(duwp_handle *h, int32_t inst, double *host_cmax, int32_t n_cells);

/* Checkpoint of the whole handle.  duwp_checkpoint_size gives the byte count; save copies the
 * complete device state into a caller-owned host buffer (synchronizing); restore loads such a
 * buffer into a handle created with identical parameters.  The generator is counter-based, so a
 * restored run continues bit-identically.  Errors: DUWP_EINVAL on size or layout mismatch. */
int duwp_checkpoint_size(duwp_handle *h, uint64_t *bytes);
int duwp_checkpoint_save(duwp_handle *h, void *host_buf, uint64_t bytes);
int duwp_checkpoint_restore(duwp_handle *h, const void *host_buf, uint64_t bytes);

/* ------------------------------------------------------------------ allocation-free inspection */

/* The paper has no counterpart: this is a library facility.  Callers that cannot allocate device
 * memory when they inspect the particles -- code running inside CUDA stream capture, where an
 * allocation would break the capture, and hosts that hand the library a fixed memory arena at
 * set-up and forbid allocations afterwards -- use this instead of duwp_get_particles.
 * Writes the particles of instance `inst`, in the same stable per-cell order and values as
 * duwp_get_particles, into caller-owned DEVICE arrays of n entries (n = duwp_num_particles):
 * cell index, cell-local position, velocity.  Asynchronous on the handle's stream; a count that
 * differs from n is recorded on the device and reported by the next synchronizing call
 * (DUWP_EOVERFLOW), and the device arrays are then left untouched.  Allocates nothing, on the
 * device or the host: the per-cell start table it needs is a static device array of
 * DUWP_NOALLOC_MAX_CELLS + 1 entries (2 MiB, held by every device that loads the library until the
 * process exits); an instance with more cells is rejected with DUWP_EINVAL.  The calling thread's
 * current device must be the handle's (DUWP_EINVAL otherwise).  The first call on a device looks
 * that array's address up and keeps it (make that first call before any stream capture).  All
 * calls share the array and each call overwrites it, so calls that overlap on the GPU (from other
 * streams or handles) race on it.  Errors: DUWP_EINVAL, DUWP_ECUDA. */
#define DUWP_NOALLOC_MAX_CELLS 262144
int duwp_get_particles_noalloc(duwp_handle *h, int32_t inst, int32_t *dev_cell, double *dev_xl,
                               double *dev_u, double *dev_v, double *dev_w, int64_t n);

/* ------------------------------------------------------------------ one instance over several parts */

/* One instance split into `parts` contiguous cell ranges of nearly equal size (part r owns cells
 * [n_cells r / parts, n_cells (r+1) / parts)), each part an engine of its own -- on the calling
 * thread's current device, or on devices[r] when `devices` (parts entries) is given -- stepped in
 * lockstep.  The method is per cell (Sec. 3.4): absorption, re-sampling and collisions act on one
 * cell's list, the transport moves particles between cells (Step 3), and the update of a cell reads
 * the wave flux of its two faces (Eq. r1).  So every step each part receives from its neighbours
 * the particles that crossed into its cells (the run of the neighbour's edge cell moving one cell
 * across, with its exact moment sums, and the farther movers with their global sort keys) and the
 * state of the neighbouring edge cell (a one-cell halo, for the flux of the boundary face and the
 * NS-corrected sampling).  Every cell then sees the list, generator ids and sums of the undivided
 * run: the results equal duwp_init's bit for bit.  The exchange goes through the host and device
 * copies (peer copies between GPUs); no kernel waits on another part.
 * Not supported (DUWP_EINVAL): periodic ends, DUWP_RECON_VANLEER (it reads two cells beyond a face).
 * Allocation as duwp_init (every part through alloc/free_fn when given).  Errors: DUWP_EINVAL,
 * DUWP_ENOMEM, DUWP_ECUDA; a run of crossing particles larger than the space reserved for it, or a
 * full far-mover list, is DUWP_EOVERFLOW from duwp_split_step. */
typedef struct duwp_split duwp_split;
int duwp_split_create(const duwp_params *params, int32_t parts, const int32_t *devices, duwp_alloc_fn alloc,
                      duwp_free_fn free_fn, void *alloc_ctx, duwp_split **out);

/* Synchronizing.  n_steps >= 0 steps of every part (Steps 1-4 of Sec. 3.4, with the exchanges).
 * Errors: DUWP_EINVAL, DUWP_ECUDA, DUWP_EOVERFLOW and the device errors of the parts. */
int duwp_split_step(duwp_split *s, int32_t n_steps);

/* Part r: its handle (owned by the split: inspect it with duwp_fields, duwp_get_particles, ...,
 * whose cell indices are local, cell i being cell c0 + i of the domain; do not step or destroy it)
 * and its cell range [c0, c1).  Any output pointer may be NULL.  Errors: DUWP_EINVAL. */
int duwp_split_part(duwp_split *s, int32_t r, duwp_handle **part, int32_t *c0, int32_t *c1);

/* Release every part. */
int duwp_split_destroy(duwp_split *s);

/* ------------------------------------------------------------------ serving (continuous batching) */

typedef struct duwp_server duwp_server;

/* hbm_budget_bytes: device memory the server may use for resident instances; max_slots: most
 * instances resident at once (per lane); max_cells: cells of the pool (per lane; 0: from the
 * budget); steps_per_launch: steps taken by all resident instances of a lane between admissions;
 * precision: record precision of every request; stream: CUDA stream of the first lane's worker;
 * lanes: 1 (or 0) one engine for every request, 2: requests of at least long_steps steps take a
 * second engine stepped on a stream of its own beside the first (the budget is split in halves). */
typedef struct {
    uint64_t hbm_budget_bytes;
    int32_t max_slots;
    int32_t max_cells;
    int32_t steps_per_launch;
    int32_t precision;
    void *stream;
    int32_t lanes;
    int32_t long_steps;
} duwp_server_cfg;

/* Result of one request.  The arrays are owned by the server and stay valid until the request
 * is released by a second duwp_poll of the same id after completion, or the server is destroyed. */
typedef struct {
    int32_t status;            /* DUWP_OK or the error that ended the request */
    int32_t n_cells;
    int64_t steps;
    int64_t particle_updates;  /* particles streamed, summed over the request's steps */
    double queue_ms;           /* submit -> admission */
    double run_ms;             /* admission -> completion */
    double step_p50_ms, step_p99_ms;  /* per-launch device time, per step */
    const double *rho, *u, *T; /* final instantaneous profile (n_cells each) */
} duwp_result;

/* Create a server with a worker thread per lane (continuous batching: requests are admitted when
 * a slot and enough of the HBM budget of their lane are free, are stepped together with every
 * request resident in their lane, and leave as soon as their own step count is reached).
 * Errors: DUWP_EINVAL (sizes, precision, lanes outside 0..2), DUWP_ENOMEM, DUWP_ECUDA. */
int duwp_server_create(const duwp_server_cfg *cfg, duwp_alloc_fn alloc, duwp_free_fn free_fn,
                       void *alloc_ctx, duwp_server **out);

/* Non-blocking: queue a request of n_steps steps; *req_id identifies it.  Errors: DUWP_EINVAL
 * (bad parameters, precision mismatch, larger than the whole budget). */
int duwp_submit(duwp_server *s, const duwp_params *params, int32_t n_steps, uint64_t *req_id);

/* Non-blocking: DUWP_PENDING while queued or running; DUWP_OK with *out filled once finished
 * (the request's own error is in out->status).  Polling a finished id a second time releases it
 * (returns DUWP_ENOTFOUND afterwards). */
int duwp_poll(duwp_server *s, uint64_t req_id, duwp_result *out);

/* Stop the worker, drop queued requests and release all memory. */
int duwp_server_destroy(duwp_server *s);

#ifdef __cplusplus
}
#endif

#endif /* DUWP_H */

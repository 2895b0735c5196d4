// duwp_launch.h -- host-side launchers of the DUWP step kernels (implemented in duwp_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "duwp_internal.cuh"

namespace duwp {

// Collision kernel of one step (direct cells of the work lists): NTC collisions in place, after the
// re-sampled particles of the cells that have any.  rp = parity of the buffer holding the arrived
// lists.  grid: persistent CTAs of collide_threads() threads.  prio: scheduling priority of the
// launch (cudaLaunchAttributePriority; a smaller number is a higher priority).
cudaError_t launch_collide(const EngineDev &E, int fp32, int rp, int grid, cudaStream_t s, int prio);
// Staged-cell kernel of one step (cells with P > 0): absorption, re-sampling and collisions into the
// staged list, one block per cell.  grid: persistent blocks (staged_occupancy() per SM).
// wide: the variant at four blocks per SM with more registers per thread (see staged_occupancy).
cudaError_t launch_staged(const EngineDev &E, int fp32, int wide, int rp, int grid, cudaStream_t s, int prio);
int staged_occupancy(int fp32, int wide);
// Particles drawn ahead of the collision kernels (direct cells with many re-sampled particles), in
// chunks over all warps: persistent blocks (sample_occupancy() per SM).
cudaError_t launch_sample(const EngineDev &E, int fp32, int rp, int grid, cudaStream_t s, int prio);
int sample_occupancy(int fp32);
// Streaming kernel of one step: one warp per cell (transport, L/S/R runs, moment sums).
cudaError_t launch_stream(const EngineDev &E, int fp32, int variant, int groups, int rp, int threads, cudaStream_t s,
                          int prio);
// Sort of the particles that moved two or more cells.
cudaError_t launch_far_sort(const EngineDev &E, int fp32, cudaStream_t s);
// Cell kernel: update Psi_t from the step's particle runs and wave flux (update = 1), then the
// primitive state, P and the slot bound of the next step (draws keyed with step index
// inst.step + (update ? 1 : 0)).  q = parity of the runs just written.
cudaError_t launch_cells(const EngineDev &E, int fp32, int q, int update, cudaStream_t s);
// Offsets of the next step's output blocks (write parity wp) and the collision work lists;
// advance = 1 also advances the per-instance step counters.
cudaError_t launch_offsets(const EngineDev &E, int wp, int advance, cudaStream_t s);
// Wave flux at every interface from the current primitive states (read by the next cell kernel).
cudaError_t launch_flux(const EngineDev &E, cudaStream_t s, int prio);
// Turn table of the double-single scattering (idempotent; once per engine).
cudaError_t launch_init_turn(cudaStream_t s);
// Initial state of the cells [g0, g0 + n) of instance b (all wave, no particles).
cudaError_t launch_init_cells(const EngineDev &E, int b, int g0, int n, const double *left_cons,
                              const double *right_cons, double x_min, double x_split, cudaStream_t s);
// The same for many instances in one launch (items by value in the kernel's parameters, at most
// kInitBatch per launch): a batch of instances is set up without a launch per instance.
struct InitCellsItem {
    double lc[5], rc[5], x_min, x_split;
    int32_t b, g0, n, pad;
};
constexpr int kInitBatch = 64;
cudaError_t launch_init_cells_batch(const EngineDev &E, const InitCellsItem *items, int n_items, cudaStream_t s);
// Profiles (rho, u, T, wave fraction) of every instance into d_out = [4 x total], instance b at
// d_base[b] (device array of n_inst entries, < 0: skip).
cudaError_t launch_moments(const EngineDev &E, int which, const int64_t *d_base, int64_t total, double *d_out,
                           cudaStream_t s);
// Normal stress and heat flux (Eq. gkt_moment1) of the interior cells among g0 .. g0 + ncell - 1:
// out[g] and out[G + g] written (accumulate = 0) or added to (accumulate = 1).  tmp: device scratch
// of stress_tmp_bytes() per flattened cell (G of them).
cudaError_t launch_stress_heat(const EngineDev &E, int fp32, int rp, int g0, int ncell, int accumulate, double *out,
                               void *tmp, cudaStream_t s);
size_t stress_tmp_bytes();
// Gather the stable sorted particle list of instance b into device arrays (debug/inspection).
// gate: NULL, or a device word that must equal `total` when the kernel runs (otherwise nothing is
// written).
cudaError_t launch_gather(const EngineDev &E, int fp32, int rp, int b, int g0, int ncell, const int64_t *d_start,
                          int64_t total, const int64_t *gate, int32_t *cell, double *xl, double *u, double *v,
                          double *w, cudaStream_t s);
// Kernel attributes (dynamic shared memory) and blocks per SM of the streaming kernel.
// variant 0: registers unconstrained (<= 128); 1: two 512-thread blocks per SM (<= 64 registers);
// 2: three (<= 40 registers); groups: 2 or 3 groups of 32 records per lane in flight
int stream_occupancy(int fp32, int variant, int groups, int threads);
size_t stream_smem_bytes(int fp32, int threads, int groups);
// The same for the collision kernel (fixed block size).
int collide_occupancy(int fp32);
size_t collide_smem_bytes(int fp32);
int collide_threads();

}  // namespace duwp

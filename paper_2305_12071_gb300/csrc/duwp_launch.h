// duwp_launch.h -- host-side launchers of the DUWP step kernels (implemented in duwp_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "duwp_internal.cuh"

namespace duwp {

// Particle kernel of one step: absorb, re-sample, collide, transport, write the L/S/R runs.
// rp = parity of the buffer holding the arrived lists.  grid: persistent CTAs.
cudaError_t launch_particles(const EngineDev &E, int fp32, int variant, int rp, int grid, int threads, size_t smem,
                             cudaStream_t s);
// Sort of the particles that moved two or more cells.
cudaError_t launch_far_sort(const EngineDev &E, int fp32, cudaStream_t s);
// Cell kernel: update Psi_t from the step's particle runs and wave flux (update = 1), then the
// primitive state, P and the slot bound of the next step (draws keyed with step index
// inst.step + (update ? 1 : 0)).  q = parity of the runs just written.
cudaError_t launch_cells(const EngineDev &E, int fp32, int q, int update, cudaStream_t s);
// Offsets of the next step's output blocks (write parity wp) and the wave flux at every
// interface; advance = 1 also advances the per-instance step counters.
cudaError_t launch_offsets_flux(const EngineDev &E, int wp, int advance, cudaStream_t s);
// Initial state of the cells [g0, g0 + n) of instance b (all wave, no particles).
cudaError_t launch_init_cells(const EngineDev &E, int b, int g0, int n, const double *left_cons,
                              const double *right_cons, double x_min, double x_split, cudaStream_t s);
// Gather the stable sorted particle list of instance b into device arrays (debug/inspection).
cudaError_t launch_gather(const EngineDev &E, int fp32, int rp, int b, int g0, int ncell, const int64_t *d_start,
                          int64_t total, int32_t *cell, double *xl, double *u, double *v, double *w, cudaStream_t s);
// Kernel attributes (dynamic shared memory) of the particle kernel; returns blocks per SM.
// variant 0: registers unconstrained; 1: capped (<= 128 threads, six blocks per SM)
int particles_occupancy(int fp32, int variant, int threads, size_t smem);
// dynamic shared memory of a particle-kernel block (one slice per warp)
size_t particles_smem_bytes(int fp32, int threads);

}  // namespace duwp

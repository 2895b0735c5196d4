// duwp_engine.h -- host-side engine: one pool of flattened cells and two particle buffers in
// HBM shared by the resident DUWP instances, stepped by one set of launches per step.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "duwp.h"
#include "duwp_internal.cuh"

namespace duwp {

void set_cuda_error(cudaError_t e, const char *where);

// Events recorded by a timed step: after the staged-cell kernel (before the collision kernel), after
// each of the five other kernels, and (last) before the staged-cell kernel.
constexpr int kStepEvents = 8;

struct HostInst {
    duwp_params p;
    InstDev d;          // constants as uploaded (step counters live on the device)
    int32_t cell_base;  // flattened index of the left reservoir cell
    double beta, lambda_ref;
    int64_t est_particles;
    bool active;
};

// Derive the constants of one instance (Sec. 4.1 Eq. lambda, Appendix A) and validate the
// description.  Returns DUWP_OK or DUWP_EINVAL.
int derive_instance(const duwp_params &p, HostInst &out);

// The same for the part of the domain of p that owns cells [c0, c1) (a domain split into cell
// ranges): global mesh, time step and generator ids; the ends that face other parts are phantom
// ends.  Errors: DUWP_EINVAL (range, periodic ends, second-order reconstruction).
int derive_part(const duwp_params &p, int32_t c0, int32_t c1, HostInst &out);

struct Engine {
    int device = 0;
    int fp32 = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    duwp_alloc_fn alloc = nullptr;
    duwp_free_fn free_fn = nullptr;
    void *alloc_ctx = nullptr;

    // sizes
    int32_t G = 0;              // flattened cells
    int32_t max_inst = 0;
    int64_t capacity = 0;       // particle slots per buffer
    int32_t far_cap = 0;
    int32_t threads = 128;      // streaming kernel: threads per block (one warp per cell)
    int32_t variant = 1;        // streaming-kernel register budget (0: <= 128, 1: <= 64, 2: <= 40 registers);
                                // the default is the autotuner's usual choice (occupancy sets the kernel's bandwidth)
    int32_t groups = 2;         // streaming kernel: groups of 32 records per lane in flight (2 or 3)
    int32_t grid_collide = 0;   // collision kernel: persistent blocks
    int32_t grid_staged = 0;    // staged-cell kernel: persistent blocks
    int32_t staged_wide = 0;    // staged-cell kernel at four blocks per SM (small pools)
    int32_t grid_sample = 0;    // drawing-ahead kernel: persistent blocks
    // one part of a split domain: the cells [part_c0, part_c1) of its single instance (part_c1 < 0:
    // not a part); pcap: slots reserved at the end of each particle buffer for the runs arriving in
    // each of the two phantom cells
    int32_t part_c0 = 0, part_c1 = -1;
    int64_t pcap = 0;

    // device memory: one slab
    void *slab = nullptr;
    size_t slab_bytes = 0;
    EngineDev dev{};
    std::vector<HostInst> inst;

    // stepping
    int parity = 0;             // parity of the buffer holding the arrived lists of the next step
    int64_t steps_done = 0;
    bool use_graphs = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // one step starting at read parity 0 / 1
    // the block kernel (cells with many collision candidates) runs beside the collision kernel (the
    // other cells) on a stream of its own, forked from and joined into the step's stream
    cudaStream_t side2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join2 = nullptr;
    cudaStream_t side3 = nullptr;                        // the wave flux beside a step's particle kernels
    cudaEvent_t ev_fork3 = nullptr, ev_join3 = nullptr;
    int prio_hi = 0, prio_lo = 0;

    // device scratch of the profile reads (allocated on first use): the table of instance bases
    // (uploaded when the set of instances changes) and two output areas of 4 x total doubles; the
    // non-blocking reads copy out on their own stream, area n_async % 2, ordered by events
    void *mom = nullptr;
    size_t mom_bytes = 0;
    size_t mom_head = 0, mom_area = 0;
    std::vector<int64_t> mom_base;
    cudaStream_t cstream = nullptr;
    cudaEvent_t mom_ready[2] = {nullptr, nullptr};
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
    int64_t n_async = 0;

    // device scratch of the stress / heat-flux read-out (allocated on first use): [Pi | Q] of the
    // last instantaneous read and [Pi | Q] running sums, G doubles each, then the per-cell
    // temporaries of the read-out passes; sums taken so far
    double *sh = nullptr;
    size_t sh_bytes = 0;
    int64_t sh_count = 0;

    ~Engine();
    int create(const duwp_params *params, int32_t n, int32_t pool_cells, int32_t pool_slots, int64_t capacity_override,
               void *stream_in, duwp_alloc_fn a, duwp_free_fn f, void *ctx);
    int configure_launch(int threads_, int variant_ = 0, int groups_ = 2);
    // used by create (upload = false: neither the table entry nor the cells yet; create copies the
    // table once and then initialises the cells) and the server
    int add_instance(int slot, const duwp_params &p, int32_t cell_base, bool upload = true);
    int init_instance_cells(int slot);
    int remove_instance(int slot);
    int enqueue_step(cudaEvent_t *ev = nullptr);   // launches of one step; ev[kStepEvents]: events around kernels
    // one third of a step's launches: 1 collisions and streaming, 2 far-mover sort and cell update,
    // 3 offsets and wave flux of the next step (and the parity flip)
    int enqueue_phase(int ph);
    int enqueue_prepare();             // cell + offset kernels without advancing (start / admission)
    // Cells the step kernels cover, [0, cells) clamped to [1, G]: every active instance must lie
    // below it and the cells above it must be unused (as remove_instance leaves them).  Drops the
    // step graphs when it changes.
    int set_run_extent(int32_t cells);
    int step(int32_t n);
    int sync();                        // wait (steps and profile copies) + read the device error word
    int moments_scratch(const std::vector<int64_t> &base, int64_t total);   // size + base table
    double *mom_out(int area) const;
    int stress_scratch();              // allocates and zeroes sh on first use
    int read_inst(int b, InstDev &out);
    void *dalloc(size_t bytes);
    void dfree(void *p, size_t bytes);
    void drop_graphs();
};

}  // namespace duwp

// The public handle: one engine.
struct duwp_handle {
    duwp::Engine eng;
};

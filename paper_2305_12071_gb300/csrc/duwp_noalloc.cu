// duwp_noalloc.cu -- particle inspection into caller-owned device arrays without any allocation.
//
// duwp_get_particles needs a table of per-cell start offsets on the device and takes it from the
// handle's allocator.  Some callers cannot allocate at that point: code running inside CUDA stream
// capture, where an allocation would break the capture, and hosts that hand the library a fixed
// memory arena at set-up and forbid allocations afterwards (embedded pipelines, frameworks that own
// the device allocator).  duwp_get_particles_noalloc keeps that table in a fixed-size array in the
// library's own device memory instead, and writes the particles straight into device arrays the
// caller provides.
#include <mutex>

#include "duwp_engine.h"
#include "duwp_launch.h"

using namespace duwp;

// Start offset of every cell of the inspected instance, followed by the instance's particle count
// (entry ncell).  Lives as long as the library is loaded, on every device that loads it (2 MiB each).
// Shared by all calls: each call overwrites the entries of the cells it handles; calls that overlap
// on the GPU race on it.
static __device__ __align__(256) int64_t g_cell_start[DUWP_NOALLOC_MAX_CELLS + 1];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int64_t *g_start_ptr[kMaxDevices] = {};

// Device address of the start table for the current device (looked up once per device).
int start_table(int device, int64_t **out)
{
    if (device < 0 || device >= kMaxDevices) return DUWP_EINVAL;
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_start_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_cell_start);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaGetSymbolAddress(g_cell_start)");
            return DUWP_ECUDA;
        }
        g_start_ptr[device] = static_cast<int64_t *>(p);
    }
    *out = g_start_ptr[device];
    return DUWP_OK;
}

// Exclusive scan of the per-cell particle counts of one instance into the start table (one block),
// the total in start[ncell]; records an overflow if the total differs from the size the caller
// passed (the gather that follows then writes nothing).
__global__ void k_start_scan(EngineDev E, int g0, int ncell, int64_t *start, int64_t expect)
{
    __shared__ int64_t s_w[32];
    __shared__ int64_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < ncell; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const int64_t v = (t < ncell) ? E.cnt[g0 + t] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        int64_t wpre = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) wpre += s_w[w];
            tot += s_w[w];
        }
        const int64_t carry = s_carry;
        if (t < ncell) start[t] = carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        start[ncell] = s_carry;
        if (s_carry != expect) atomicCAS(E.err, 0, -7);
    }
}

}  // namespace

extern "C" int duwp_get_particles_noalloc(duwp_handle *h, int32_t inst, int32_t *dev_cell, double *dev_xl,
                                          double *dev_u, double *dev_v, double *dev_w, int64_t n)
{
    if (!h) return DUWP_EINVAL;
    Engine &E = h->eng;
    if (inst < 0 || inst >= E.max_inst || !E.inst[inst].active) return DUWP_EINVAL;
    const HostInst &hi = E.inst[inst];
    const int32_t C = hi.p.n_cells;
    if (C > DUWP_NOALLOC_MAX_CELLS) return DUWP_EINVAL;
    if (n < 0 || (n > 0 && (!dev_cell || !dev_xl || !dev_u || !dev_v || !dev_w))) return DUWP_EINVAL;
    // the table of the handle's device: the symbol's address is looked up with that device current
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaGetDevice");
        return DUWP_ECUDA;
    }
    if (device != E.device) return DUWP_EINVAL;
    int64_t *start = nullptr;
    const int rc = start_table(device, &start);
    if (rc != DUWP_OK) return rc;
    k_start_scan<<<1, 1024, 0, E.stream>>>(E.dev, hi.cell_base + 1, C, start, n);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_gather(E.dev, E.fp32, E.parity, inst, hi.cell_base + 1, C, start, n, start + C, dev_cell, dev_xl,
                          dev_u, dev_v, dev_w, E.stream);
    if (e != cudaSuccess) {
        set_cuda_error(e, "duwp_get_particles_noalloc");
        return DUWP_ECUDA;
    }
    return DUWP_OK;
}

// duwp_api.cu -- host side of the DUWP library: problem validation and derived constants
// (Sec. 4.1 Eq. lambda, Appendix A), the engine (one HBM pool of cells and particle buffers
// stepped by one set of launches per step, captured in CUDA graphs), inspection, checkpoints,
// and the C ABI declared in include/duwp.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "duwp_engine.h"
#include "duwp_launch.h"

namespace duwp {

static thread_local std::string g_last_cuda;

void set_cuda_error(cudaError_t e, const char *where)
{
    g_last_cuda = std::string(where) + ": " + cudaGetErrorString(e);
}

#define DUWP_CU(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            set_cuda_error(e_, #call);                  \
            return DUWP_ECUDA;                          \
        }                                               \
    } while (0)

static bool finite_state(const duwp_state &s) { return std::isfinite(s.rho) && std::isfinite(s.u) && std::isfinite(s.v) && std::isfinite(s.w) && std::isfinite(s.T); }

static void cons_of(const duwp_state &s, double R, double *c)
{
    c[0] = s.rho;
    c[1] = s.rho * s.u;
    c[2] = s.rho * s.v;
    c[3] = s.rho * s.w;
    c[4] = 0.5 * s.rho * (s.u * s.u + s.v * s.v + s.w * s.w) + 1.5 * s.rho * R * s.T;
}

int derive_instance(const duwp_params &p, HostInst &o)
{
    if (p.n_cells < 1 || p.n_cells > (1 << 26)) return DUWP_EINVAL;
    if (!(p.x_max > p.x_min) || !(p.ppc_ref > 0.0) || !(p.Kn > 0.0) || !(p.L_ref > 0.0)) return DUWP_EINVAL;
    if (!(p.R > 0.0) || !(p.Pr > 0.0) || !(p.rho_ref > 0.0) || !(p.T_ref > 0.0) || !(p.alpha > 0.0)) return DUWP_EINVAL;
    if (!(p.omega >= 0.5 && p.omega <= 1.0)) return DUWP_EINVAL;
    if (!finite_state(p.left) || !finite_state(p.right)) return DUWP_EINVAL;
    if (p.left.rho < 0.0 || p.right.rho < 0.0 || !(p.left.T > 0.0) || !(p.right.T > 0.0)) return DUWP_EINVAL;
    for (int32_t bc : {p.bc_left, p.bc_right})
        if (bc < 0 || bc > 3) return DUWP_EINVAL;
    if ((p.bc_left == DUWP_BC_PERIODIC) != (p.bc_right == DUWP_BC_PERIODIC)) return DUWP_EINVAL;
    if (p.precision != DUWP_FP64 && p.precision != DUWP_FP32) return DUWP_EINVAL;
    if (p.eps_mode < 0 || p.eps_mode > 3 || p.flux_mode < 0 || p.flux_mode > 1 || p.ntc_rate < 0 || p.ntc_rate > 1)
        return DUWP_EINVAL;
    if (p.resample_mode != DUWP_RESAMPLE_MAXWELL && p.resample_mode != DUWP_RESAMPLE_CE) return DUWP_EINVAL;
    if (p.split_mode != DUWP_SPLIT_P && p.split_mode != DUWP_SPLIT_QMC) return DUWP_EINVAL;
    if (p.recon_mode != DUWP_RECON_FIRST && p.recon_mode != DUWP_RECON_VANLEER) return DUWP_EINVAL;
    if (!(p.dt > 0.0) && !(p.cfl > 0.0)) return DUWP_EINVAL;

    o.p = p;
    InstDev &d = o.d;
    std::memset(&d, 0, sizeof d);
    d.C = p.n_cells;
    d.bc_left = p.bc_left;
    d.bc_right = p.bc_right;
    d.eps_mode = p.eps_mode;
    d.flux_mode = p.flux_mode;
    d.ntc_rate = p.ntc_rate;
    d.resample_mode = p.resample_mode;
    d.split_mode = p.split_mode;
    d.recon_mode = p.recon_mode;
    d.active = 1;
    d.key0 = static_cast<uint32_t>(p.seed & 0xffffffffu);
    d.key1 = static_cast<uint32_t>(p.seed >> 32);
    d.step = 0;
    d.avg_start = p.avg_start;
    d.navg = 0;
    d.dx = (p.x_max - p.x_min) / static_cast<double>(p.n_cells);
    // Eq. (lambda), first form, solved for the viscosity at the reference state
    o.beta = 5.0 * (p.alpha + 1.0) * (p.alpha + 2.0) / (4.0 * p.alpha * (5.0 - 2.0 * p.omega) * (7.0 - 2.0 * p.omega));
    o.lambda_ref = p.Kn * p.L_ref;
    const double p_ref = p.rho_ref * p.R * p.T_ref;
    d.mu_ref = o.beta * o.lambda_ref * p_ref * std::sqrt(2.0 * kPi / (p.R * p.T_ref));
    d.mp = p.rho_ref * d.dx / p.ppc_ref;
    d.dx_over_mp = d.dx / d.mp;
    d.mp_over_dx = d.mp / d.dx;
    if (p.dt > 0.0) {
        d.dt = p.dt;
    } else {
        const double sl = std::fabs(p.left.u) + 3.0 * std::sqrt(2.0 * p.R * p.left.T);
        const double sr = std::fabs(p.right.u) + 3.0 * std::sqrt(2.0 * p.R * p.right.T);
        d.dt = p.cfl * d.dx / std::max(sl, sr);
    }
    if (!(d.dt > 0.0) || !std::isfinite(d.dt)) return DUWP_EINVAL;
    d.dtdx = d.dt / d.dx;
    d.dtdx_f = static_cast<float>(d.dtdx);
    d.R = p.R;
    d.Pr = p.Pr;
    d.omega = p.omega;
    d.T_ref = p.T_ref;
    d.rho_ref = p.rho_ref;
    d.upsilon = p.omega - 0.5;
    // reference relative speed of the VHS cross-section: sqrt(2kT_ref/m_r) / Gamma(2.5-omega)^{0.5/upsilon},
    // 2kT_ref/m_r = 4 R T_ref for equal masses (Appendix A)
    if (d.upsilon == 0.0) d.c_ref = std::sqrt(4.0 * p.R * p.T_ref);
    else d.c_ref = std::sqrt(4.0 * p.R * p.T_ref) / std::pow(std::tgamma(2.5 - p.omega), 0.5 / d.upsilon);
    d.ntc_A = d.dt / (2.0 * std::sqrt(2.0) * o.lambda_ref);
    d.ntc_rr = (d.mp / d.dx) / p.rho_ref;
    d.inv_rho_ref = 1.0 / p.rho_ref;
    d.inv_cv = 1.0 / (1.5 * p.R);
    d.vhs_expo = 1.0 - 2.0 * d.upsilon;
    d.vhs_expo_f = static_cast<float>(d.vhs_expo);
    d.mu_ref_f = static_cast<float>(d.mu_ref);
    d.T_ref_f = static_cast<float>(d.T_ref);
    d.omega_f = static_cast<float>(d.omega);
    d.R_f = static_cast<float>(d.R);
    d.dt_f = static_cast<float>(d.dt);
    const duwp_state *st[2] = {&p.left, &p.right};
    for (int s = 0; s < 2; ++s) {
        double *q = s ? d.right : d.left;
        q[0] = st[s]->rho; q[1] = st[s]->u; q[2] = st[s]->v; q[3] = st[s]->w; q[4] = st[s]->T;
    }
    // particles expected from the initial mass (a capacity estimate): the cells whose centre lies
    // left of x_split are a prefix, found by bisection with the same test as the cell set-up
    int32_t lo = 0, hi = p.n_cells;
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        const double xc = p.x_min + (static_cast<double>(mid) + 0.5) * d.dx;
        if (xc < p.x_split) lo = mid + 1;
        else hi = mid;
    }
    const double mass = (static_cast<double>(lo) * p.left.rho + static_cast<double>(p.n_cells - lo) * p.right.rho) * d.dx;
    o.est_particles = static_cast<int64_t>(std::ceil(mass / d.mp));
    o.active = true;
    return DUWP_OK;
}

int derive_part(const duwp_params &p, int32_t c0, int32_t c1, HostInst &o)
{
    if (c0 < 0 || c1 > p.n_cells || c0 >= c1) return DUWP_EINVAL;
    // the split keeps the undivided order between non-periodic ends, with one phantom cell per side
    // (first-order interface states of the wave flux)
    if (p.bc_left == DUWP_BC_PERIODIC || p.recon_mode != DUWP_RECON_FIRST) return DUWP_EINVAL;
    const int rc = derive_instance(p, o);
    if (rc != DUWP_OK) return rc;
    o.p.n_cells = c1 - c0;
    o.d.C = c1 - c0;
    o.d.id0 = c0;
    if (c0 > 0) o.d.bc_left = kBcPhantom;
    if (c1 < p.n_cells) o.d.bc_right = kBcPhantom;
    double mass = 0.0;
    for (int32_t i = c0; i < c1; ++i) {
        const double xc = p.x_min + (static_cast<double>(i) + 0.5) * o.d.dx;
        mass += (xc < p.x_split ? p.left.rho : p.right.rho) * o.d.dx;
    }
    o.est_particles = static_cast<int64_t>(std::ceil(mass / o.d.mp));
    return DUWP_OK;
}

// ------------------------------------------------------------------------------------------
// Engine
// ------------------------------------------------------------------------------------------
void *Engine::dalloc(size_t bytes)
{
    if (alloc && free_fn) return alloc(bytes, stream, alloc_ctx);
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaMallocAsync");
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Engine::dfree(void *p, size_t bytes)
{
    if (!p) return;
    if (alloc && free_fn) free_fn(p, bytes, stream, alloc_ctx);
    else cudaFreeAsync(p, stream);
}

void Engine::drop_graphs()
{
    for (auto &gx : graph) {
        if (gx) cudaGraphExecDestroy(gx);
        gx = nullptr;
    }
}

Engine::~Engine()
{
    if (cstream) cudaStreamSynchronize(cstream);
    if (stream) cudaStreamSynchronize(stream);
    drop_graphs();
    if (side2) cudaStreamSynchronize(side2);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join2) cudaEventDestroy(ev_join2);
    if (side3) cudaStreamSynchronize(side3);
    if (ev_fork3) cudaEventDestroy(ev_fork3);
    if (ev_join3) cudaEventDestroy(ev_join3);
    if (side3) cudaStreamDestroy(side3);
    if (side2) cudaStreamDestroy(side2);
    for (int k = 0; k < 2; ++k) {
        if (mom_ready[k]) cudaEventDestroy(mom_ready[k]);
        if (copy_done[k]) cudaEventDestroy(copy_done[k]);
    }
    if (cstream) cudaStreamDestroy(cstream);
    if (mom) dfree(mom, mom_bytes);
    if (sh) dfree(sh, sh_bytes);
    dfree(slab, slab_bytes);
    if (stream) cudaStreamSynchronize(stream);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

namespace {
struct Carver {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count)
    {
        off = (off + 255) & ~static_cast<size_t>(255);
        const size_t o = off;
        off += count * sizeof(T);
        return o;
    }
};
}  // namespace

int Engine::configure_launch(int threads_, int variant_, int groups_)
{
    if (threads_ < 32 || threads_ > 512 || (threads_ & 31)) return DUWP_EINVAL;
    if (variant_ < 0 || variant_ > 2 || groups_ < 2 || groups_ > 3) return DUWP_EINVAL;
    const int occ = stream_occupancy(fp32, variant_, groups_, threads_);
    if (occ <= 0) return DUWP_EINVAL;
    const int occ_c = collide_occupancy(fp32);
    if (occ_c <= 0) return DUWP_EINVAL;
    const int occ_p = sample_occupancy(fp32);
    if (occ_p <= 0) return DUWP_EINVAL;
    int nsm = 0;
    DUWP_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    // block kernel: a small pool (at most 8 cells per SM, so that its heavy cells fit in one wave at
    // four blocks per SM) takes the variant with more registers per thread; a larger one keeps five
    // blocks per SM in flight (measured: one 1000-cell Sod tube 0.163 -> 0.154 ms per step, 25 tubes
    // 0.479 -> 0.488 ms)
    staged_wide = (static_cast<int64_t>(G) <= 8 * static_cast<int64_t>(nsm)) ? 1 : 0;
    const int occ_s = staged_occupancy(fp32, staged_wide);
    if (occ_s <= 0) return DUWP_EINVAL;
    dev.nsm = nsm;
    threads = threads_;
    variant = variant_;
    groups = groups_;
    // collision kernel: persistent blocks, as many as fit, but no more warps than cells
    const int cw = collide_threads() / 32;
    grid_collide = std::max(1, std::min(occ_c * nsm, (G + cw - 1) / cw));
    // staged-cell kernel: one block per cell, as many persistent blocks as fit, no more than cells
    grid_staged = std::max(1, std::min(occ_s * nsm, G));
    grid_sample = std::max(1, occ_p * nsm);
    drop_graphs();
    return DUWP_OK;
}

int Engine::create(const duwp_params *params, int32_t n, int32_t pool_cells, int32_t pool_slots, int64_t cap_override,
                   void *stream_in, duwp_alloc_fn a, duwp_free_fn f, void *ctx)
{
    alloc = a;
    free_fn = f;
    alloc_ctx = ctx;
    DUWP_CU(cudaGetDevice(&device));
    if (stream_in) {
        stream = static_cast<cudaStream_t>(stream_in);
    } else {
        DUWP_CU(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
        own_stream = true;
    }
    if (!params || n < 0) return DUWP_EINVAL;
    DUWP_CU(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    DUWP_CU(cudaStreamCreateWithFlags(&side2, cudaStreamNonBlocking));
    DUWP_CU(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    DUWP_CU(cudaEventCreateWithFlags(&ev_join2, cudaEventDisableTiming));
    DUWP_CU(cudaStreamCreateWithFlags(&side3, cudaStreamNonBlocking));
    DUWP_CU(cudaEventCreateWithFlags(&ev_fork3, cudaEventDisableTiming));
    DUWP_CU(cudaEventCreateWithFlags(&ev_join3, cudaEventDisableTiming));
    std::vector<HostInst> hs(static_cast<size_t>(n));
    int64_t est = 0;
    int64_t cells = 0;
    double max_ppc = 0.0;
    if (part_c1 >= 0 && n != 1) return DUWP_EINVAL;
    for (int32_t b = 0; b < n; ++b) {
        const int rc = (part_c1 >= 0) ? derive_part(params[b], part_c0, part_c1, hs[b]) : derive_instance(params[b], hs[b]);
        if (rc != DUWP_OK) return rc;
        if (params[b].precision != params[0].precision) return DUWP_EINVAL;
        est += hs[b].est_particles;
        cells += hs[b].p.n_cells + 2;
        const double rmax = std::max(params[b].left.rho, params[b].right.rho) / params[b].rho_ref;
        max_ppc = std::max(max_ppc, rmax * params[b].ppc_ref);
    }
    fp32 = (params[0].precision == DUWP_FP32) ? 1 : 0;
    if (pool_cells > 0) cells = std::max<int64_t>(cells, pool_cells);
    if (cells > (int64_t(1) << 30)) return DUWP_EINVAL;
    G = static_cast<int32_t>(cells);
    max_inst = std::max<int32_t>(n, pool_slots);
    if (max_inst < 1) return DUWP_EINVAL;
    // particle slots: every cell's output block is twice its slot bound, and the slot bound is at
    // most twice the cell's mass in particles (plus 2) in the re-sampling regimes
    int64_t cap = 4 * est + 8 * static_cast<int64_t>(G) + 8192;
    uint64_t cap_user = 0;
    for (int32_t b = 0; b < n; ++b) cap_user = std::max<uint64_t>(cap_user, params[b].capacity);
    if (cap_override > 0) cap = cap_override;
    else if (cap_user > 0) cap = static_cast<int64_t>(cap_user);
    if (cap >= (int64_t(1) << 40)) return DUWP_EINVAL;
    capacity = cap;

    far_cap = 1 << 16;

    const size_t rec = fp32 ? sizeof(RecF) : sizeof(RecD);
    const size_t far_item = fp32 ? sizeof(FarItem<RecF>) : sizeof(FarItem<RecD>);
    const int32_t nblocks = (G + kCellBlockMin - 1) / kCellBlockMin;   // blocks of the cell kernels at their smallest
    Carver c;
    const size_t o_inst = c.take<InstDev>(max_inst);
    const size_t o_cinst = c.take<int32_t>(G);
    const size_t o_psi = c.take<double>(5 * size_t(G));
    const size_t o_prim = c.take<double>(5 * size_t(G));
    const size_t o_valid = c.take<int32_t>(G);
    const size_t o_P = c.take<double>(G);
    const size_t o_cmax = c.take<double>(G);
    const size_t o_fmaj = c.take<double>(G);
    const size_t o_flux = c.take<double>(5 * size_t(G));
    const size_t o_avg = c.take<double>(5 * size_t(G));
    const size_t o_AL = c.take<int64_t>(4 * size_t(G));
    const size_t o_AR = c.take<int64_t>(4 * size_t(G));
    const size_t o_As = c.take<int64_t>(5 * size_t(G));
    const size_t o_slots = c.take<int32_t>(G);
    const size_t o_cnt = c.take<int32_t>(G);
    size_t o_nL[2], o_nS[2], o_nR[2], o_off[2];
    size_t o_sb[2];
    for (int p = 0; p < 2; ++p) {
        o_sb[p] = c.take<int32_t>(G);
        o_nL[p] = c.take<int32_t>(G);
        o_nS[p] = c.take<int32_t>(G);
        o_nR[p] = c.take<int32_t>(G);
        o_off[p] = c.take<int64_t>(G);
    }
    const size_t o_bs = c.take<int64_t>(nblocks);
    const size_t o_nnew = c.take<int32_t>(G), o_nabs = c.take<int32_t>(G), o_ncand = c.take<int32_t>(G),
                 o_nacc = c.take<int32_t>(G);
    const size_t o_fc = c.take<int32_t>(4);
    const size_t o_err = c.take<int32_t>(4);
    const size_t o_ticket = c.take<int32_t>(kTickets);
    const size_t o_hdr = c.take<CellHdr>(G);
    const size_t o_wl = c.take<int32_t>(kLists * size_t(G));
    // chunks of re-sampled particles: at most one partial chunk per cell plus the re-sampled
    // particles (at most half the slots of a buffer) in full chunks
    const int64_t wls_cap = int64_t(G) + capacity / (2 * kSampleChunk) + 64;
    if (wls_cap > INT32_MAX) return DUWP_EINVAL;
    const size_t o_wls = c.take<int2>(size_t(wls_cap));
    const size_t o_wlp = c.take<int2>(size_t(wls_cap));
    const size_t o_wr = c.take<int2>(size_t(G));
    const size_t o_wgrp = c.take<int2>(size_t(G) / 32 + 1);
    const size_t o_wlnc = c.take<int32_t>(size_t(G));
    const size_t o_fa = c.take<unsigned char>(far_item * far_cap);
    const size_t o_fs = c.take<unsigned char>(far_item * far_cap);
    // each buffer: the output blocks, then (one part of a split domain) the runs arriving in its two
    // phantom cells from the neighbouring parts
    if (part_c1 >= 0) pcap = 2 * ((4 * static_cast<int64_t>(std::ceil(max_ppc)) + 1024) / 2);
    const size_t o_buf0 = c.take<unsigned char>(rec * size_t(capacity + 2 * pcap));
    const size_t o_buf1 = c.take<unsigned char>(rec * size_t(capacity + 2 * pcap));
    slab_bytes = (c.off + 255) & ~static_cast<size_t>(255);
    slab = dalloc(slab_bytes);
    if (!slab) return DUWP_ENOMEM;
    unsigned char *base = static_cast<unsigned char *>(slab);
    // zero everything except the particle buffers, then mark all cells unused
    DUWP_CU(cudaMemsetAsync(base, 0, o_buf0, stream));
    dev.G = G;
    dev.G_run = G;
    dev.n_inst = max_inst;
    dev.capacity = capacity;
    dev.far_cap = far_cap;
    dev.inst = reinterpret_cast<InstDev *>(base + o_inst);
    dev.cell_inst = reinterpret_cast<int32_t *>(base + o_cinst);
    dev.psi = reinterpret_cast<double *>(base + o_psi);
    dev.prim = reinterpret_cast<double *>(base + o_prim);
    dev.valid = reinterpret_cast<int32_t *>(base + o_valid);
    dev.P = reinterpret_cast<double *>(base + o_P);
    dev.cmax = reinterpret_cast<double *>(base + o_cmax);
    dev.fmaj = reinterpret_cast<double *>(base + o_fmaj);
    dev.flux = reinterpret_cast<double *>(base + o_flux);
    dev.avg = reinterpret_cast<double *>(base + o_avg);
    dev.AL = reinterpret_cast<int64_t *>(base + o_AL);
    dev.AR = reinterpret_cast<int64_t *>(base + o_AR);
    dev.Aself = reinterpret_cast<int64_t *>(base + o_As);
    dev.slots = reinterpret_cast<int32_t *>(base + o_slots);
    dev.cnt = reinterpret_cast<int32_t *>(base + o_cnt);
    for (int p = 0; p < 2; ++p) {
        dev.slotsb[p] = reinterpret_cast<int32_t *>(base + o_sb[p]);
        dev.nL[p] = reinterpret_cast<int32_t *>(base + o_nL[p]);
        dev.nS[p] = reinterpret_cast<int32_t *>(base + o_nS[p]);
        dev.nR[p] = reinterpret_cast<int32_t *>(base + o_nR[p]);
        dev.off[p] = reinterpret_cast<int64_t *>(base + o_off[p]);
    }
    dev.blocksum = reinterpret_cast<int64_t *>(base + o_bs);
    dev.nnew = reinterpret_cast<int32_t *>(base + o_nnew);
    dev.nabs = reinterpret_cast<int32_t *>(base + o_nabs);
    dev.ncand = reinterpret_cast<int32_t *>(base + o_ncand);
    dev.nacc = reinterpret_cast<int32_t *>(base + o_nacc);
    dev.far_count = reinterpret_cast<int32_t *>(base + o_fc);
    dev.err = reinterpret_cast<int32_t *>(base + o_err);
    dev.ticket = reinterpret_cast<int32_t *>(base + o_ticket);
    dev.hdr = reinterpret_cast<CellHdr *>(base + o_hdr);
    dev.wl = reinterpret_cast<int32_t *>(base + o_wl);
    dev.wls = reinterpret_cast<int2 *>(base + o_wls);
    dev.wlp = reinterpret_cast<int2 *>(base + o_wlp);
    dev.wr = reinterpret_cast<int2 *>(base + o_wr);
    dev.wgrp = reinterpret_cast<int2 *>(base + o_wgrp);
    dev.wlnc = reinterpret_cast<int32_t *>(base + o_wlnc);
    dev.wls_cap = static_cast<int32_t>(wls_cap);
    dev.far_app = base + o_fa;
    dev.far_sorted = base + o_fs;
    dev.buf[0] = base + o_buf0;
    dev.buf[1] = base + o_buf1;
    DUWP_CU(cudaMemsetAsync(dev.cell_inst, 0xff, sizeof(int32_t) * size_t(G), stream));
    DUWP_CU(launch_init_turn(stream));

    int rc = configure_launch(threads, variant, groups);
    if (rc != DUWP_OK) return rc;

    inst.assign(static_cast<size_t>(max_inst), HostInst{});
    for (auto &h : inst) h.active = false;
    int32_t gb = 0;
    for (int32_t b = 0; b < n; ++b) {
        rc = add_instance(b, params[b], gb, false);
        if (rc != DUWP_OK) return rc;
        gb += inst[b].p.n_cells + 2;
    }
    // the instance table in one copy (a copy from pageable memory waits for the stream), then the
    // cells of every instance
    if (n > 0) {
        std::vector<InstDev> table(static_cast<size_t>(n));
        for (int32_t b = 0; b < n; ++b) table[b] = inst[b].d;
        DUWP_CU(cudaMemcpyAsync(dev.inst, table.data(), sizeof(InstDev) * static_cast<size_t>(n), cudaMemcpyHostToDevice,
                                stream));
        DUWP_CU(cudaStreamSynchronize(stream));
        // every instance's cells in one launch per kInitBatch instances
        std::vector<InitCellsItem> items(static_cast<size_t>(n));
        for (int32_t b = 0; b < n; ++b) {
            const duwp_params &p = inst[b].p;
            InitCellsItem &q = items[static_cast<size_t>(b)];
            cons_of(p.left, p.R, q.lc);
            cons_of(p.right, p.R, q.rc);
            q.x_min = p.x_min;
            q.x_split = p.x_split;
            q.b = b;
            q.g0 = inst[b].cell_base;
            q.n = p.n_cells + 2;
            q.pad = 0;
        }
        DUWP_CU(launch_init_cells_batch(dev, items.data(), n, stream));
    }
    rc = enqueue_prepare();
    if (rc != DUWP_OK) return rc;
    return sync();
}

int Engine::add_instance(int slot, const duwp_params &p, int32_t cell_base, bool upload)
{
    if (slot < 0 || slot >= max_inst) return DUWP_EINVAL;
    HostInst h;
    int rc = (part_c1 >= 0) ? derive_part(p, part_c0, part_c1, h) : derive_instance(p, h);
    if (rc != DUWP_OK) return rc;
    if ((p.precision == DUWP_FP32) != (fp32 == 1)) return DUWP_EINVAL;
    if (cell_base < 0 || int64_t(cell_base) + h.p.n_cells + 2 > G) return DUWP_EINVAL;
    h.cell_base = cell_base;
    h.d.cell_base = cell_base;
    inst[slot] = h;
    if (!upload) return DUWP_OK;
    DUWP_CU(cudaMemcpyAsync(dev.inst + slot, &inst[slot].d, sizeof(InstDev), cudaMemcpyHostToDevice, stream));
    return init_instance_cells(slot);
}

int Engine::init_instance_cells(int slot)
{
    const duwp_params &p = inst[slot].p;
    double lc[5], rc5[5];
    cons_of(p.left, p.R, lc);
    cons_of(p.right, p.R, rc5);
    DUWP_CU(launch_init_cells(dev, slot, inst[slot].cell_base, p.n_cells + 2, lc, rc5, p.x_min, p.x_split, stream));
    return DUWP_OK;
}

int Engine::remove_instance(int slot)
{
    if (slot < 0 || slot >= max_inst || !inst[slot].active) return DUWP_EINVAL;
    const HostInst &h = inst[slot];
    DUWP_CU(cudaMemsetAsync(dev.cell_inst + h.cell_base, 0xff, sizeof(int32_t) * size_t(h.p.n_cells + 2), stream));
    DUWP_CU(cudaMemsetAsync(dev.slots + h.cell_base, 0, sizeof(int32_t) * size_t(h.p.n_cells + 2), stream));
    // class kClsSkip (0) until the next cell kernel rebuilds the plans
    DUWP_CU(cudaMemsetAsync(dev.hdr + h.cell_base, 0, sizeof(CellHdr) * size_t(h.p.n_cells + 2), stream));
    inst[slot].active = false;
    return DUWP_OK;
}

int Engine::set_run_extent(int32_t cells)
{
    const int32_t n = std::max<int32_t>(1, std::min(cells, G));
    if (n == dev.G_run) return DUWP_OK;
    // the grids of the captured step graphs follow the extent
    dev.G_run = n;
    drop_graphs();
    return DUWP_OK;
}

int Engine::enqueue_prepare()
{
    // Recompute the primitive state, P, slot bounds and offsets of every cell from the current state
    // without advancing: idempotent for instances already running (same inputs and draws), and the
    // start of a newly added one.  (The wave flux is formed at the start of the next step.)
    DUWP_CU(launch_cells(dev, fp32, parity, 0, stream));
    DUWP_CU(launch_offsets(dev, 1 - parity, 0, stream));
    return DUWP_OK;
}

int Engine::enqueue_phase(int ph)
{
    const int rp = parity;
    if (ph == 1) {
        // the wave flux of the states of the last cell kernel, on a third stream beside the
        // particle kernels; the cell kernel of phase 2 waits for it
        DUWP_CU(cudaEventRecord(ev_fork3, stream));
        DUWP_CU(cudaStreamWaitEvent(side3, ev_fork3, 0));
        DUWP_CU(launch_flux(dev, side3, prio_hi));
        DUWP_CU(cudaEventRecord(ev_join3, side3));
        // the block kernel (cells with many candidates, which draw their own re-sampled particles)
        // on a second stream from the start; beside it the light cells' rounds and the particles
        // drawn ahead, then the collision kernel (the other cells that need one); then every cell
        // streams in one launch.  (Streaming the cells that need no collision beside the collision
        // kernels was 1.6% slower on the bench batch once the collision kernel had become short.)
        DUWP_CU(cudaStreamWaitEvent(side2, ev_fork3, 0));
        DUWP_CU(launch_staged(dev, fp32, staged_wide, rp, grid_staged, side2, prio_hi));
        DUWP_CU(cudaEventRecord(ev_join2, side2));
        DUWP_CU(launch_sample(dev, fp32, rp, grid_sample, stream, prio_hi));
        DUWP_CU(launch_collide(dev, fp32, rp, grid_collide, stream, prio_hi));
        DUWP_CU(cudaStreamWaitEvent(stream, ev_join2, 0));
        DUWP_CU(launch_stream(dev, fp32, variant, groups, rp, threads, stream, prio_hi));
    } else if (ph == 2) {
        DUWP_CU(launch_far_sort(dev, fp32, stream));
        DUWP_CU(cudaStreamWaitEvent(stream, ev_join3, 0));
        DUWP_CU(launch_cells(dev, fp32, 1 - rp, 1, stream));
    } else {
        DUWP_CU(launch_offsets(dev, rp, 1, stream));
        parity = 1 - rp;
    }
    return DUWP_OK;
}

int Engine::enqueue_step(cudaEvent_t *ev)
{
    const int rp = parity;
    if (!ev) {
        for (int ph = 1; ph <= 3; ++ph) {
            const int rc = enqueue_phase(ph);
            if (rc != DUWP_OK) return rc;
        }
        return DUWP_OK;
    }
    {
        // timed: one kernel after the other, events around each (ev[7]: before the wave flux)
        DUWP_CU(cudaEventRecord(ev[7], stream));
        DUWP_CU(launch_flux(dev, stream, prio_hi));
        DUWP_CU(cudaEventRecord(ev[6], stream));
        DUWP_CU(launch_sample(dev, fp32, rp, grid_sample, stream, prio_hi));
        DUWP_CU(launch_staged(dev, fp32, staged_wide, rp, grid_staged, stream, prio_hi));
        DUWP_CU(cudaEventRecord(ev[0], stream));
        DUWP_CU(launch_collide(dev, fp32, rp, grid_collide, stream, prio_hi));
        DUWP_CU(cudaEventRecord(ev[1], stream));
        DUWP_CU(launch_stream(dev, fp32, variant, groups, rp, threads, stream, prio_hi));
        DUWP_CU(cudaEventRecord(ev[2], stream));
    }
    DUWP_CU(launch_far_sort(dev, fp32, stream));
    DUWP_CU(cudaEventRecord(ev[3], stream));
    DUWP_CU(launch_cells(dev, fp32, 1 - rp, 1, stream));
    DUWP_CU(cudaEventRecord(ev[4], stream));
    DUWP_CU(launch_offsets(dev, rp, 1, stream));
    DUWP_CU(cudaEventRecord(ev[5], stream));
    parity = 1 - rp;
    return DUWP_OK;
}

int Engine::step(int32_t n)
{
    if (n < 0) return DUWP_EINVAL;
    int32_t left = n;
    if (use_graphs) {
        while (left >= 1) {
            // one graph per read parity, each holding the launches of one step
            const int p0 = parity;
            cudaGraphExec_t &gx = graph[p0];
            if (!gx) {
                cudaGraph_t gr = nullptr;
                DUWP_CU(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
                const int rc = enqueue_step();
                cudaError_t e = cudaStreamEndCapture(stream, &gr);
                parity = p0;
                if (rc != DUWP_OK) return rc;
                if (e != cudaSuccess) { set_cuda_error(e, "cudaStreamEndCapture"); return DUWP_ECUDA; }
                e = cudaGraphInstantiate(&gx, gr, cudaGraphInstantiateFlagUseNodePriority);
                cudaGraphDestroy(gr);
                if (e != cudaSuccess) { set_cuda_error(e, "cudaGraphInstantiate"); gx = nullptr; return DUWP_ECUDA; }
            }
            DUWP_CU(cudaGraphLaunch(gx, stream));
            parity = 1 - p0;
            left -= 1;
            steps_done += 1;
        }
    }
    while (left > 0) {
        const int rc = enqueue_step();
        if (rc != DUWP_OK) return rc;
        --left;
        ++steps_done;
    }
    return DUWP_OK;
}

int Engine::sync()
{
    if (cstream) DUWP_CU(cudaStreamSynchronize(cstream));
    // (the flux stream's work is joined into the step's stream before the cell kernel; synchronized
    // here too for a sequence of phases cut short by an error)
    if (side3) DUWP_CU(cudaStreamSynchronize(side3));
    DUWP_CU(cudaStreamSynchronize(stream));
    int32_t e = 0;
    DUWP_CU(cudaMemcpy(&e, dev.err, sizeof e, cudaMemcpyDeviceToHost));
    return e;
}

int Engine::read_inst(int b, InstDev &out)
{
    DUWP_CU(cudaMemcpyAsync(&out, dev.inst + b, sizeof(InstDev), cudaMemcpyDeviceToHost, stream));
    DUWP_CU(cudaStreamSynchronize(stream));
    return DUWP_OK;
}

}  // namespace duwp

using namespace duwp;

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

const char *duwp_error_string(int s)
{
    switch (s) {
    case DUWP_OK: return "ok";
    case DUWP_EINVAL: return "invalid argument or problem description";
    case DUWP_ENOMEM: return "allocation failed";
    case DUWP_ECUDA: return "CUDA error";
    case DUWP_ENUMERIC: return "non-finite or non-physical state";
    case DUWP_ETIMEOUT: return "bounded device wait ran out";
    case DUWP_EBUSY: return "busy: cannot admit now";
    case DUWP_EOVERFLOW: return "cell, particle-buffer or far-mover overflow";
    case DUWP_ENOTFOUND: return "unknown request id";
    case DUWP_PENDING: return "pending";
    default: return "unknown status";
    }
}

const char *duwp_last_cuda_error(void) { return g_last_cuda.c_str(); }

int duwp_init_batch(const duwp_params *params, int32_t n, void *stream, duwp_alloc_fn alloc, duwp_free_fn free_fn,
                    void *alloc_ctx, duwp_handle **out)
{
    if (!params || n < 1 || !out) return DUWP_EINVAL;
    *out = nullptr;
    duwp_handle *h = new (std::nothrow) duwp_handle;
    if (!h) return DUWP_ENOMEM;
    const int rc = h->eng.create(params, n, 0, 0, 0, stream, alloc, free_fn, alloc_ctx);
    if (rc != DUWP_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return DUWP_OK;
}

int duwp_init(const duwp_params *params, void *stream, duwp_alloc_fn alloc, duwp_free_fn free_fn, void *alloc_ctx,
              duwp_handle **out)
{
    return duwp_init_batch(params, 1, stream, alloc, free_fn, alloc_ctx, out);
}

int duwp_step(duwp_handle *h, int32_t n_steps)
{
    if (!h) return DUWP_EINVAL;
    return h->eng.step(n_steps);
}

int duwp_sync(duwp_handle *h)
{
    if (!h) return DUWP_EINVAL;
    return h->eng.sync();
}

int duwp_step_timed(duwp_handle *h, int32_t n, double *kernel_ms, double *step_ms)
{
    if (!h || n < 1 || !kernel_ms) return DUWP_EINVAL;
    Engine &E = h->eng;
    constexpr int kEv = kStepEvents;
    std::vector<cudaEvent_t> ev(kEv * static_cast<size_t>(n), nullptr);
    int rc = DUWP_OK;
    for (auto &e : ev) {
        if (cudaEventCreate(&e) != cudaSuccess) { rc = DUWP_ECUDA; break; }
    }
    for (int32_t s = 0; s < n && rc == DUWP_OK; ++s) {
        rc = E.enqueue_step(ev.data() + kEv * static_cast<size_t>(s));
        if (rc == DUWP_OK) ++E.steps_done;
    }
    if (rc == DUWP_OK) rc = E.sync();
    for (int k = 0; k < DUWP_TIMED_SLOTS; ++k) kernel_ms[k] = 0.0;
    if (rc == DUWP_OK) {
        // per step: e[7] before the wave flux, e[6] before the staged-cell kernel, e[0] before the
        // collision kernel, e[1..5] after the collision, streaming, far-sort, cell and offset kernels
        float span = 0.f;
        cudaEventElapsedTime(&span, ev[7], ev[kEv * static_cast<size_t>(n - 1) + 5]);
        kernel_ms[5] = span;
        for (int32_t s = 0; s < n; ++s) {
            cudaEvent_t *e = ev.data() + kEv * static_cast<size_t>(s);
            for (int k = 0; k < 5; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e[k], e[k + 1]);
                kernel_ms[k] += ms;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e[6], e[0]);
            kernel_ms[6] += ms;
            cudaEventElapsedTime(&ms, e[7], e[6]);     // the wave flux, with the offsets in [4]
            kernel_ms[4] += ms;
            if (step_ms) {
                cudaEventElapsedTime(&ms, e[7], e[5]);
                step_ms[s] = ms;
            }
        }
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    return rc;
}

int duwp_shock_normalise(int32_t kind, int64_t n, const double *x, const double *rho, const double *T, const double *Pi,
                         const double *Q, double rho_up, double T_up, double rho_down, double T_down, double lam_up,
                         double beta, double R, double *x_out, double *rho_out, double *T_out, double *Pi_out,
                         double *Q_out)
{
    if ((kind != DUWP_SHOCK_MA3 && kind != DUWP_SHOCK_MA8) || n < 0) return DUWP_EINVAL;
    if ((x_out && !x) || (rho_out && !rho) || (T_out && !T) || (Pi_out && !Pi) || (Q_out && !Q)) return DUWP_EINVAL;
    if (!(rho_up > 0.0) || !(T_up > 0.0) || !(lam_up > 0.0) || !(R > 0.0)) return DUWP_EINVAL;
    const double p_up = rho_up * R * T_up, s = 2.0 * R * T_up;
    double xs, r0, rs, t0, ts, ps, qs;
    if (kind == DUWP_SHOCK_MA3) {
        xs = 0.5 * std::sqrt(kPi) * lam_up;
        r0 = 0.0; rs = rho_up;
        t0 = 0.0; ts = T_up;
        ps = p_up;
        qs = p_up * std::sqrt(s);
    } else {
        if (!(beta > 0.0) || rho_down == rho_up || T_down == T_up) return DUWP_EINVAL;
        xs = beta * kPi * lam_up;
        r0 = rho_up; rs = rho_down - rho_up;
        t0 = T_up; ts = T_down - T_up;
        ps = rho_up * s;
        qs = rho_up * s * std::sqrt(s);
    }
    for (int64_t i = 0; i < n; ++i) {
        if (x_out) x_out[i] = x[i] / xs;
        if (rho_out) rho_out[i] = (rho[i] - r0) / rs;
        if (T_out) T_out[i] = (T[i] - t0) / ts;
        if (Pi_out) Pi_out[i] = Pi[i] / ps;
        if (Q_out) Q_out[i] = Q[i] / qs;
    }
    return DUWP_OK;
}

int duwp_destroy(duwp_handle *h)
{
    if (!h) return DUWP_EINVAL;
    delete h;
    return DUWP_OK;
}

static int check_inst(duwp_handle *h, int32_t b)
{
    if (!h || b < 0 || b >= h->eng.max_inst || !h->eng.inst[b].active) return DUWP_EINVAL;
    return DUWP_OK;
}

int duwp_fields(duwp_handle *h, int32_t b, int32_t which, double *host_psi, int32_t n, int64_t *host_navg)
{
    int rc = check_inst(h, b);
    if (rc) return rc;
    Engine &E = h->eng;
    const HostInst &hi = E.inst[b];
    if (n != hi.p.n_cells || !host_psi || (which != DUWP_INSTANT && which != DUWP_AVERAGED)) return DUWP_EINVAL;
    rc = E.sync();
    if (rc) return rc;
    const double *src = (which == DUWP_INSTANT ? E.dev.psi : E.dev.avg) + 5 * size_t(hi.cell_base + 1);
    DUWP_CU(cudaMemcpy(host_psi, src, sizeof(double) * 5 * size_t(n), cudaMemcpyDeviceToHost));
    InstDev d;
    rc = E.read_inst(b, d);
    if (rc) return rc;
    if (host_navg) *host_navg = d.navg;
    return DUWP_OK;
}

int duwp_moments(duwp_handle *h, int32_t b, int32_t which, double *rho, double *u, double *T, double *wave_frac,
                 int32_t n)
{
    int rc = check_inst(h, b);
    if (rc) return rc;
    Engine &E = h->eng;
    const HostInst &hi = E.inst[b];
    if (n != hi.p.n_cells) return DUWP_EINVAL;
    std::vector<double> psi(5 * static_cast<size_t>(n));
    int64_t navg = 0;
    rc = duwp_fields(h, b, which, psi.data(), n, &navg);
    if (rc) return rc;
    std::vector<int32_t> cnt(static_cast<size_t>(n), 0);
    DUWP_CU(cudaMemcpy(cnt.data(), E.dev.cnt + hi.cell_base + 1, sizeof(int32_t) * size_t(n), cudaMemcpyDeviceToHost));
    std::vector<double> cur(5 * static_cast<size_t>(n));
    if (wave_frac) DUWP_CU(cudaMemcpy(cur.data(), E.dev.psi + 5 * size_t(hi.cell_base + 1), sizeof(double) * 5 * size_t(n), cudaMemcpyDeviceToHost));
    const double scale = (which == DUWP_AVERAGED) ? (navg > 0 ? 1.0 / static_cast<double>(navg) : 0.0) : 1.0;
    for (int32_t i = 0; i < n; ++i) {
        const double *c = psi.data() + 5 * size_t(i);
        // the same arithmetic as the all-instance read-out kernel (one reciprocal per density)
        const double r = c[0] * scale;
        const double mx = c[1] * scale, my = c[2] * scale, mz = c[3] * scale, E5 = c[4] * scale;
        const double ir = r > 0 ? 1.0 / r : 0.0;
        const double ux = mx * ir, uy = my * ir, uz = mz * ir;
        const double tt = r > 0 ? (E5 * ir - 0.5 * (ux * ux + uy * uy + uz * uz)) * hi.d.inv_cv : 0.0;
        if (rho) rho[i] = r;
        if (u) u[i] = ux;
        if (T) T[i] = tt;
        if (wave_frac) {
            const double rt = cur[5 * size_t(i)];
            const double irt = (which == DUWP_AVERAGED) ? (rt > 0 ? 1.0 / rt : 0.0) : ir;
            wave_frac[i] = rt > 0 ? 1.0 - (static_cast<double>(cnt[i]) * hi.d.mp_over_dx) * irt : 0.0;
        }
    }
    return DUWP_OK;
}

namespace duwp {

int Engine::stress_scratch()
{
    if (sh) return DUWP_OK;
    const size_t bytes = (4 * sizeof(double) + stress_tmp_bytes()) * size_t(G);
    sh = static_cast<double *>(dalloc(bytes));
    if (!sh) return DUWP_ENOMEM;
    sh_bytes = bytes;
    sh_count = 0;
    DUWP_CU(cudaMemsetAsync(sh, 0, 4 * sizeof(double) * size_t(G), stream));
    return DUWP_OK;
}

int Engine::moments_scratch(const std::vector<int64_t> &base, int64_t total)
{
    const size_t head = (sizeof(int64_t) * base.size() + 255) & ~static_cast<size_t>(255);
    const size_t area = (sizeof(double) * 4 * static_cast<size_t>(total) + 255) & ~static_cast<size_t>(255);
    const size_t need = head + 2 * area;
    if (mom_bytes >= need && base == mom_base && mom_area == area) return DUWP_OK;
    // the scratch may still be read by pending copies: wait for them first
    int rc = sync();
    if (rc) return rc;
    if (mom_bytes < need) {
        if (mom) dfree(mom, mom_bytes);
        mom = nullptr;
        mom_bytes = 0;
        mom = dalloc(need);
        if (!mom) return DUWP_ENOMEM;
        mom_bytes = need;
    }
    mom_head = head;
    mom_area = area;
    DUWP_CU(cudaMemcpyAsync(mom, base.data(), sizeof(int64_t) * base.size(), cudaMemcpyHostToDevice, stream));
    DUWP_CU(cudaStreamSynchronize(stream));
    mom_base = base;
    return DUWP_OK;
}

double *Engine::mom_out(int area) const
{
    return reinterpret_cast<double *>(static_cast<unsigned char *>(mom) + mom_head + static_cast<size_t>(area) * mom_area);
}

}  // namespace duwp

// Bases of the active instances' cells in the output arrays of the profile reads; returns the total.
static int64_t moment_bases(const Engine &E, std::vector<int64_t> &base)
{
    base.assign(static_cast<size_t>(E.max_inst), -1);
    int64_t total = 0;
    for (int32_t b = 0; b < E.max_inst; ++b) {
        if (!E.inst[b].active) continue;
        base[b] = total;
        total += E.inst[b].p.n_cells;
    }
    return total;
}

int duwp_moments_all(duwp_handle *h, int32_t which, double *rho, double *u, double *T, double *wave_frac,
                     int64_t total_cells)
{
    if (!h || (which != DUWP_INSTANT && which != DUWP_AVERAGED)) return DUWP_EINVAL;
    Engine &E = h->eng;
    std::vector<int64_t> base;
    const int64_t total = moment_bases(E, base);
    if (total != total_cells) return DUWP_EINVAL;
    if (total == 0) return E.sync();
    int rc = E.moments_scratch(base, total);
    if (rc) return rc;
    // area 0 may be the target of a pending non-blocking read
    if (E.cstream) DUWP_CU(cudaStreamSynchronize(E.cstream));
    double *d_out = E.mom_out(0);
    DUWP_CU(launch_moments(E.dev, which, static_cast<const int64_t *>(E.mom), total, d_out, E.stream));
    double *dst[4] = {rho, u, T, wave_frac};
    for (int k = 0; k < 4; ++k)
        if (dst[k])
            DUWP_CU(cudaMemcpyAsync(dst[k], d_out + static_cast<size_t>(k) * total, sizeof(double) * total,
                                    cudaMemcpyDeviceToHost, E.stream));
    return E.sync();
}

int duwp_moments_all_async(duwp_handle *h, int32_t which, double *rho, double *u, double *T, double *wave_frac,
                           int64_t total_cells)
{
    if (!h || (which != DUWP_INSTANT && which != DUWP_AVERAGED)) return DUWP_EINVAL;
    Engine &E = h->eng;
    std::vector<int64_t> base;
    const int64_t total = moment_bases(E, base);
    if (total != total_cells) return DUWP_EINVAL;
    if (total == 0) return DUWP_OK;
    int rc = E.moments_scratch(base, total);
    if (rc) return rc;
    if (!E.cstream) {
        DUWP_CU(cudaStreamCreateWithFlags(&E.cstream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            DUWP_CU(cudaEventCreateWithFlags(&E.mom_ready[k], cudaEventDisableTiming));
            DUWP_CU(cudaEventCreateWithFlags(&E.copy_done[k], cudaEventDisableTiming));
        }
    }
    const int a = static_cast<int>(E.n_async & 1);
    // area a is free once the copies of the read two calls back have finished
    if (E.n_async >= 2) DUWP_CU(cudaStreamWaitEvent(E.stream, E.copy_done[a], 0));
    double *d_out = E.mom_out(a);
    DUWP_CU(launch_moments(E.dev, which, static_cast<const int64_t *>(E.mom), total, d_out, E.stream));
    DUWP_CU(cudaEventRecord(E.mom_ready[a], E.stream));
    DUWP_CU(cudaStreamWaitEvent(E.cstream, E.mom_ready[a], 0));
    double *dst[4] = {rho, u, T, wave_frac};
    for (int k = 0; k < 4; ++k)
        if (dst[k])
            DUWP_CU(cudaMemcpyAsync(dst[k], d_out + static_cast<size_t>(k) * total, sizeof(double) * total,
                                    cudaMemcpyDeviceToHost, E.cstream));
    DUWP_CU(cudaEventRecord(E.copy_done[a], E.cstream));
    E.n_async += 1;
    return DUWP_OK;
}

int duwp_moments_wait(duwp_handle *h)
{
    if (!h) return DUWP_EINVAL;
    Engine &E = h->eng;
    if (E.cstream) DUWP_CU(cudaStreamSynchronize(E.cstream));
    return DUWP_OK;
}

int duwp_get_info(duwp_handle *h, int32_t b, duwp_info *out)
{
    int rc = check_inst(h, b);
    if (rc || !out) return DUWP_EINVAL;
    Engine &E = h->eng;
    const HostInst &hi = E.inst[b];
    out->dx = hi.d.dx;
    out->dt = hi.d.dt;
    out->mp = hi.d.mp;
    out->beta = hi.beta;
    out->lambda_ref = hi.lambda_ref;
    out->mu_ref = hi.d.mu_ref;
    out->c_ref = hi.d.c_ref;
    out->capacity = E.capacity;
    int ni = 0;
    for (const auto &x : E.inst) ni += x.active ? 1 : 0;
    out->n_instances = ni;
    InstDev d;
    rc = E.read_inst(b, d);
    if (rc) return rc;
    out->steps_done = d.step;
    out->particle_updates = static_cast<int64_t>(d.updates);
    return DUWP_OK;
}

int duwp_set_launch(duwp_handle *h, int32_t threads, int32_t reg_capped, int32_t groups)
{
    if (!h) return DUWP_EINVAL;
    Engine &E = h->eng;
    const int rc = E.sync();
    if (rc) return rc;
    return E.configure_launch(threads, reg_capped, groups);
}

int duwp_use_graphs(duwp_handle *h, int32_t on)
{
    if (!h) return DUWP_EINVAL;
    h->eng.use_graphs = on != 0;
    return DUWP_OK;
}

int duwp_num_particles(duwp_handle *h, int32_t b, int64_t *out)
{
    int rc = check_inst(h, b);
    if (rc || !out) return DUWP_EINVAL;
    Engine &E = h->eng;
    rc = E.sync();
    if (rc) return rc;
    const HostInst &hi = E.inst[b];
    std::vector<int32_t> cnt(static_cast<size_t>(hi.p.n_cells));
    DUWP_CU(cudaMemcpy(cnt.data(), E.dev.cnt + hi.cell_base + 1, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost));
    int64_t s = 0;
    for (int32_t c : cnt) s += c;
    *out = s;
    return DUWP_OK;
}

int duwp_get_particles(duwp_handle *h, int32_t b, int32_t *cell, double *xl, double *u, double *v, double *w, int64_t n)
{
    int64_t np = 0;
    int rc = duwp_num_particles(h, b, &np);
    if (rc) return rc;
    if (n != np || !cell || !xl || !u || !v || !w) return DUWP_EINVAL;
    Engine &E = h->eng;
    const HostInst &hi = E.inst[b];
    const int32_t C = hi.p.n_cells;
    std::vector<int32_t> cnt(static_cast<size_t>(C));
    DUWP_CU(cudaMemcpy(cnt.data(), E.dev.cnt + hi.cell_base + 1, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> start(static_cast<size_t>(C));
    int64_t s = 0;
    for (int32_t i = 0; i < C; ++i) { start[i] = s; s += cnt[i]; }
    const size_t nb = std::max<int64_t>(np, 1);
    const size_t bytes = sizeof(int64_t) * size_t(C) + nb * (sizeof(int32_t) + 4 * sizeof(double)) + 1024;
    unsigned char *tmp = static_cast<unsigned char *>(E.dalloc(bytes));
    if (!tmp) return DUWP_ENOMEM;
    int64_t *d_start = reinterpret_cast<int64_t *>(tmp);
    double *d_xl = reinterpret_cast<double *>(tmp + ((sizeof(int64_t) * size_t(C) + 255) & ~size_t(255)));
    double *d_u = d_xl + nb, *d_v = d_u + nb, *d_w = d_v + nb;
    int32_t *d_cell = reinterpret_cast<int32_t *>(d_w + nb);
    cudaError_t e = cudaMemcpyAsync(d_start, start.data(), sizeof(int64_t) * size_t(C), cudaMemcpyHostToDevice, E.stream);
    if (e == cudaSuccess) e = launch_gather(E.dev, E.fp32, E.parity, b, hi.cell_base + 1, C, d_start, np, nullptr, d_cell, d_xl, d_u, d_v, d_w, E.stream);
    if (e == cudaSuccess && np > 0) {
        e = cudaMemcpyAsync(cell, d_cell, sizeof(int32_t) * size_t(np), cudaMemcpyDeviceToHost, E.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(xl, d_xl, sizeof(double) * size_t(np), cudaMemcpyDeviceToHost, E.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, d_u, sizeof(double) * size_t(np), cudaMemcpyDeviceToHost, E.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(v, d_v, sizeof(double) * size_t(np), cudaMemcpyDeviceToHost, E.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w, d_w, sizeof(double) * size_t(np), cudaMemcpyDeviceToHost, E.stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    E.dfree(tmp, bytes);
    if (e != cudaSuccess) { set_cuda_error(e, "duwp_get_particles"); return DUWP_ECUDA; }
    return E.sync();
}

int duwp_stress_heat(duwp_handle *h, int32_t b, int32_t which, double *Pi, double *Q, int32_t n)
{
    int rc = check_inst(h, b);
    if (rc) return rc;
    if (which != DUWP_INSTANT && which != DUWP_AVERAGED) return DUWP_EINVAL;
    Engine &E = h->eng;
    const HostInst &hi = E.inst[b];
    if (n != hi.p.n_cells || !Pi || !Q) return DUWP_EINVAL;
    rc = E.stress_scratch();
    if (rc) return rc;
    const int32_t g0 = hi.cell_base + 1;
    const double *src = E.sh + (which == DUWP_INSTANT ? 0 : 2 * size_t(E.G));
    cudaError_t e = cudaSuccess;
    if (which == DUWP_INSTANT) e = launch_stress_heat(E.dev, E.fp32, E.parity, g0, n, 0, E.sh, E.sh + 4 * size_t(E.G), E.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Pi, src + g0, sizeof(double) * size_t(n), cudaMemcpyDeviceToHost, E.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Q, src + E.G + g0, sizeof(double) * size_t(n), cudaMemcpyDeviceToHost, E.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) { set_cuda_error(e, "duwp_stress_heat"); return DUWP_ECUDA; }
    rc = E.sync();
    if (rc) return rc;
    if (which == DUWP_AVERAGED) {
        const double scale = E.sh_count > 0 ? 1.0 / static_cast<double>(E.sh_count) : 0.0;
        for (int32_t i = 0; i < n; ++i) { Pi[i] *= scale; Q[i] *= scale; }
    }
    return DUWP_OK;
}

int duwp_stress_heat_accumulate(duwp_handle *h)
{
    if (!h) return DUWP_EINVAL;
    Engine &E = h->eng;
    const int rc = E.stress_scratch();
    if (rc) return rc;
    DUWP_CU(launch_stress_heat(E.dev, E.fp32, E.parity, 0, E.dev.G_run, 1, E.sh + 2 * size_t(E.G), E.sh + 4 * size_t(E.G), E.stream));
    E.sh_count += 1;
    return DUWP_OK;
}

int duwp_get_counters(duwp_handle *h, int32_t b, int32_t *ncand, int32_t *nacc, int32_t *nabs, int32_t *nnew, int32_t n)
{
    int rc = check_inst(h, b);
    if (rc) return rc;
    Engine &E = h->eng;
    const HostInst &hi = E.inst[b];
    if (n != hi.p.n_cells) return DUWP_EINVAL;
    rc = E.sync();
    if (rc) return rc;
    const size_t o = size_t(hi.cell_base + 1), by = sizeof(int32_t) * size_t(n);
    if (ncand) DUWP_CU(cudaMemcpy(ncand, E.dev.ncand + o, by, cudaMemcpyDeviceToHost));
    if (nacc) DUWP_CU(cudaMemcpy(nacc, E.dev.nacc + o, by, cudaMemcpyDeviceToHost));
    if (nabs) DUWP_CU(cudaMemcpy(nabs, E.dev.nabs + o, by, cudaMemcpyDeviceToHost));
    if (nnew) DUWP_CU(cudaMemcpy(nnew, E.dev.nnew + o, by, cudaMemcpyDeviceToHost));
    return DUWP_OK;
}

int duwp_get_cmax(duwp_handle *h, int32_t b, double *cmax, int32_t n)
{
    int rc = check_inst(h, b);
    if (rc) return rc;
    Engine &E = h->eng;
    const HostInst &hi = E.inst[b];
    if (n != hi.p.n_cells || !cmax) return DUWP_EINVAL;
    rc = E.sync();
    if (rc) return rc;
    DUWP_CU(cudaMemcpy(cmax, E.dev.cmax + hi.cell_base + 1, sizeof(double) * size_t(n), cudaMemcpyDeviceToHost));
    return DUWP_OK;
}

struct CkptHeader {
    uint64_t magic, slab_bytes, capacity;
    int32_t G, max_inst, fp32, parity;
    int64_t steps_done;
};
static const uint64_t kCkptMagic = 0x4455575043503031ull;

int duwp_checkpoint_size(duwp_handle *h, uint64_t *bytes)
{
    if (!h || !bytes) return DUWP_EINVAL;
    *bytes = sizeof(CkptHeader) + h->eng.slab_bytes;
    return DUWP_OK;
}

int duwp_checkpoint_save(duwp_handle *h, void *buf, uint64_t bytes)
{
    if (!h || !buf) return DUWP_EINVAL;
    Engine &E = h->eng;
    if (bytes != sizeof(CkptHeader) + E.slab_bytes) return DUWP_EINVAL;
    const int rc = E.sync();
    if (rc) return rc;
    CkptHeader hd{kCkptMagic, E.slab_bytes, static_cast<uint64_t>(E.capacity), E.G, E.max_inst, E.fp32, E.parity, E.steps_done};
    std::memcpy(buf, &hd, sizeof hd);
    DUWP_CU(cudaMemcpy(static_cast<unsigned char *>(buf) + sizeof hd, E.slab, E.slab_bytes, cudaMemcpyDeviceToHost));
    return DUWP_OK;
}

int duwp_checkpoint_restore(duwp_handle *h, const void *buf, uint64_t bytes)
{
    if (!h || !buf) return DUWP_EINVAL;
    Engine &E = h->eng;
    if (bytes != sizeof(CkptHeader) + E.slab_bytes) return DUWP_EINVAL;
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kCkptMagic || hd.slab_bytes != E.slab_bytes || hd.G != E.G || hd.max_inst != E.max_inst ||
        hd.fp32 != E.fp32 || hd.capacity != static_cast<uint64_t>(E.capacity))
        return DUWP_EINVAL;
    DUWP_CU(cudaStreamSynchronize(E.stream));
    DUWP_CU(cudaMemcpy(E.slab, static_cast<const unsigned char *>(buf) + sizeof hd, E.slab_bytes, cudaMemcpyHostToDevice));
    E.parity = hd.parity;
    E.steps_done = hd.steps_done;
    return E.sync();
}

}  // extern "C"

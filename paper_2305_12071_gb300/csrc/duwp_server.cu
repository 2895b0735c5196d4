// duwp_server.cu -- continuous-batching server of DUWP solves over one or two engines (lanes).
//
// Requests (a problem description and a step count) queue on the host.  A worker thread owns each
// lane's engine: between launches it admits queued requests while an instance slot, a contiguous
// range of pool cells and enough of the particle-slot budget are free (admission by HBM footprint),
// steps every resident request of the lane together (one set of launches over the occupied part of
// the cell pool, replayed from CUDA graphs, so requests admitted meanwhile join the next launch),
// and retires each request as soon as its own step count is reached: its profile is copied out, its
// cells and slots freed.  With two lanes, requests of many steps (at least long_steps) take the
// second engine, which steps on its own stream beside the first at a higher scheduling priority:
// their many steps then cost their own lane's step time rather than that of every short request
// resident meanwhile.  Each request
// draws only from its own generator key, so its result does not depend on what else is resident
// or on its lane.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "duwp_engine.h"
#include "duwp_launch.h"

using namespace duwp;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    duwp_params p{};
    int32_t n_steps = 0;
    int64_t reserve = 0;      // particle slots reserved in the buffers
    int32_t slot = -1, cell_base = -1;
    int64_t done_steps = 0;
    int64_t updates0 = 0;
    Clock::time_point t_submit, t_admit, t_done;
    std::vector<double> step_ms;
    int32_t status = DUWP_OK;
    std::vector<double> rho, u, T;
    bool finished = false;
};

// First-fit allocator of contiguous cell ranges in the pool.
struct RangeAlloc {
    std::map<int32_t, int32_t> free_;   // start -> length
    void init(int32_t n) { free_.clear(); free_[0] = n; }
    int32_t take(int32_t n)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const int32_t s = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[s + n] = len - n;
                return s;
            }
        }
        return -1;
    }
    void give(int32_t s, int32_t n)
    {
        auto it = free_.emplace(s, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const size_t k = std::min(v.size() - 1, static_cast<size_t>(std::ceil(q * v.size())) - (q > 0 ? 1 : 0));
    return v[k];
}

}  // namespace

// One lane: an engine with its own stream and worker thread, the requests resident on it, its free
// cell ranges and the particle slots reserved.  Lanes step concurrently on the device.
struct Lane {
    Engine eng;
    std::thread worker;
    std::deque<Request *> queue;
    std::vector<Request *> resident;     // indexed by instance slot
    RangeAlloc cells;
    int64_t reserved = 0;
    int32_t engine_error = DUWP_OK;
};

struct duwp_server {
    duwp_server_cfg cfg{};
    std::vector<Lane *> lanes;           // lane 0: short requests; lane 1 (if any): long requests
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_id = 1;
    std::map<uint64_t, Request *> all;

    int64_t footprint(const HostInst &h) const
    {
        return 4 * h.est_particles + 8 * static_cast<int64_t>(h.p.n_cells + 2) + 64;
    }
    int lane_of(int32_t n_steps) const
    {
        return (lanes.size() > 1 && cfg.long_steps > 0 && n_steps >= cfg.long_steps) ? 1 : 0;
    }

    void run(Lane &L);
    bool admit_locked(Lane &L);
    void retire(Lane &L, Request *r);
    static int32_t run_extent(const Lane &L);
};

// Cells the step kernels cover: up to the end of the highest resident range, rounded up to a
// granule so that small changes keep the captured graphs (first-fit keeps the ranges low, and an
// empty pool's cells cost block launches every step).
int32_t duwp_server::run_extent(const Lane &L)
{
    constexpr int32_t kGranule = 4096;
    int32_t hi = 0;
    for (const Request *r : L.resident)
        if (r) hi = std::max(hi, r->cell_base + r->p.n_cells + 2);
    return ((hi + kGranule - 1) / kGranule) * kGranule;
}

void duwp_server::retire(Lane &L, Request *r)
{
    Engine &eng = L.eng;
    const HostInst &hi = eng.inst[r->slot];
    const int32_t n = hi.p.n_cells;
    std::vector<double> psi(5 * static_cast<size_t>(n));
    r->rho.assign(static_cast<size_t>(n), 0.0);
    r->u.assign(static_cast<size_t>(n), 0.0);
    r->T.assign(static_cast<size_t>(n), 0.0);
    cudaError_t e = cudaMemcpyAsync(psi.data(), eng.dev.psi + 5 * static_cast<size_t>(hi.cell_base + 1),
                                    sizeof(double) * psi.size(), cudaMemcpyDeviceToHost, eng.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(eng.stream);
    if (e != cudaSuccess) {
        set_cuda_error(e, "server result copy");
        r->status = DUWP_ECUDA;
    }
    for (int32_t i = 0; i < n; ++i) {
        const double *c = psi.data() + 5 * static_cast<size_t>(i);
        // the same arithmetic as the library's other read-outs (one reciprocal per density)
        const double rho = c[0];
        const double ir = rho > 0 ? 1.0 / rho : 0.0;
        const double ux = c[1] * ir, uy = c[2] * ir, uz = c[3] * ir;
        r->rho[i] = rho;
        r->u[i] = ux;
        r->T[i] = rho > 0 ? (c[4] * ir - 0.5 * (ux * ux + uy * uy + uz * uz)) * hi.d.inv_cv : 0.0;
    }
    eng.remove_instance(r->slot);
    L.cells.give(r->cell_base, n + 2);
    L.resident[r->slot] = nullptr;
    L.reserved -= r->reserve;
    r->t_done = Clock::now();
    r->finished = true;
}

bool duwp_server::admit_locked(Lane &L)
{
    Engine &eng = L.eng;
    bool any = false;
    while (!L.queue.empty()) {
        Request *r = L.queue.front();
        int32_t slot = -1;
        for (int32_t s = 0; s < eng.max_inst; ++s)
            if (!L.resident[s]) { slot = s; break; }
        if (slot < 0 || L.reserved + r->reserve > eng.capacity) break;
        const int32_t base = L.cells.take(r->p.n_cells + 2);
        if (base < 0) break;
        const int rc = eng.add_instance(slot, r->p, base);
        L.queue.pop_front();
        if (rc != DUWP_OK) {
            L.cells.give(base, r->p.n_cells + 2);
            r->status = rc;
            r->finished = true;
            r->t_admit = r->t_done = Clock::now();
            continue;
        }
        r->slot = slot;
        r->cell_base = base;
        r->t_admit = Clock::now();
        L.resident[slot] = r;
        L.reserved += r->reserve;
        any = true;
    }
    return any;
}

void duwp_server::run(Lane &L)
{
    Engine &eng = L.eng;
    cudaSetDevice(eng.device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        const bool admitted = admit_locked(L);
        int32_t n_res = 0;
        int64_t min_left = INT64_MAX;
        for (Request *r : L.resident) {
            if (!r) continue;
            ++n_res;
            min_left = std::min<int64_t>(min_left, r->n_steps - r->done_steps);
        }
        if (n_res == 0) {
            cv.wait(lk, [&] { return stop || !L.queue.empty(); });
            continue;
        }
        const int32_t extent = run_extent(L);
        lk.unlock();
        int rc = DUWP_OK;
        if (admitted) {
            rc = eng.set_run_extent(extent);
            if (rc == DUWP_OK) rc = eng.enqueue_prepare();
        }
        const int32_t k = static_cast<int32_t>(std::min<int64_t>(std::max(1, cfg.steps_per_launch), min_left));
        float ms = 0.f;
        if (rc == DUWP_OK && k > 0) {
            cudaEventRecord(e0, eng.stream);
            rc = eng.step(k);
            cudaEventRecord(e1, eng.stream);
            if (rc == DUWP_OK) rc = eng.sync();
            cudaEventElapsedTime(&ms, e0, e1);
        }
        lk.lock();
        if (rc != DUWP_OK) L.engine_error = rc;
        for (Request *r : L.resident) {
            if (!r) continue;
            if (k > 0) {
                r->done_steps += k;
                for (int32_t s = 0; s < k; ++s) r->step_ms.push_back(ms / k);
            }
            if (rc != DUWP_OK) r->status = rc;
        }
        bool retired = false;
        for (Request *r : std::vector<Request *>(L.resident)) {
            if (!r) continue;
            if (r->done_steps >= r->n_steps || r->status != DUWP_OK) {
                InstDev d;
                if (eng.read_inst(r->slot, d) == DUWP_OK) r->updates0 = static_cast<int64_t>(d.updates);
                retire(L, r);
                retired = true;
            }
        }
        if (retired) {
            eng.set_run_extent(run_extent(L));
            lk.unlock();
            const int rc2 = eng.enqueue_prepare();
            lk.lock();
            if (rc2 != DUWP_OK) L.engine_error = rc2;
        }
        cv.notify_all();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

extern "C" {

int duwp_server_create(const duwp_server_cfg *cfg, duwp_alloc_fn alloc, duwp_free_fn free_fn, void *alloc_ctx,
                       duwp_server **out)
{
    if (!cfg || !out || cfg->max_slots < 1 || cfg->hbm_budget_bytes == 0) return DUWP_EINVAL;
    if (cfg->precision != DUWP_FP32 && cfg->precision != DUWP_FP64) return DUWP_EINVAL;
    if (cfg->lanes < 0 || cfg->lanes > 2 || cfg->long_steps < 0) return DUWP_EINVAL;
    *out = nullptr;
    duwp_server *s = new (std::nothrow) duwp_server;
    if (!s) return DUWP_ENOMEM;
    s->cfg = *cfg;
    const int n_lanes = std::max(1, cfg->lanes);
    // pool: cells given, or 1/64 of the budget at ~400 bytes per cell of per-cell state; with two
    // lanes each takes half of the budget (and of the cells and slots)
    int64_t cells = cfg->max_cells > 0 ? cfg->max_cells : static_cast<int64_t>(cfg->hbm_budget_bytes / 64 / 400);
    cells = std::max<int64_t>(cells, 1024);
    cells = std::min<int64_t>(cells, int64_t(1) << 26);
    const int64_t rec = cfg->precision == DUWP_FP32 ? 16 : 32;
    const int64_t per_cell = 420;
    const int64_t budget = static_cast<int64_t>(cfg->hbm_budget_bytes) / n_lanes;
    int64_t left = budget - cells * per_cell - (int64_t(16) << 20);
    if (left <= 0) { delete s; return DUWP_EINVAL; }
    const int64_t cap = left / (2 * rec);
    for (int l = 0; l < n_lanes; ++l) {
        Lane *L = new (std::nothrow) Lane;
        if (!L) { duwp_server_destroy(s); return DUWP_ENOMEM; }
        s->lanes.push_back(L);
        // the engine is created empty: a placeholder description fixes the precision only; lane 0
        // steps on the caller's stream, lane 1 on a stream of its own
        duwp_params dummy{};
        dummy.precision = cfg->precision;
        const int rc = L->eng.create(&dummy, 0, static_cast<int32_t>(cells), cfg->max_slots, cap,
                                     l == 0 ? cfg->stream : nullptr, alloc, free_fn, alloc_ctx);
        if (rc != DUWP_OK) { duwp_server_destroy(s); return rc; }
        L->resident.assign(static_cast<size_t>(L->eng.max_inst), nullptr);
        L->cells.init(L->eng.G);
        // with two lanes the short lane's kernels take the lowest scheduling priority: the long
        // requests, whose many steps set the tail of the latency, are placed first
        if (n_lanes > 1 && l == 0) L->eng.prio_hi = L->eng.prio_lo;
    }
    for (Lane *L : s->lanes) L->worker = std::thread([s, L] { s->run(*L); });
    *out = s;
    return DUWP_OK;
}

int duwp_submit(duwp_server *s, const duwp_params *params, int32_t n_steps, uint64_t *req_id)
{
    if (!s || !params || !req_id || n_steps < 1) return DUWP_EINVAL;
    HostInst h;
    int rc = derive_instance(*params, h);
    if (rc != DUWP_OK) return rc;
    if ((params->precision == DUWP_FP32) != (s->lanes[0]->eng.fp32 == 1)) return DUWP_EINVAL;
    Request *r = new (std::nothrow) Request;
    if (!r) return DUWP_ENOMEM;
    r->p = *params;
    r->n_steps = n_steps;
    r->reserve = s->footprint(h);
    r->t_submit = Clock::now();
    Lane &L = *s->lanes[s->lane_of(n_steps)];
    if (r->reserve > L.eng.capacity || params->n_cells + 2 > L.eng.G) {
        delete r;
        return DUWP_EINVAL;
    }
    std::lock_guard<std::mutex> g(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    L.queue.push_back(r);
    *req_id = r->id;
    s->cv.notify_all();
    return DUWP_OK;
}

int duwp_poll(duwp_server *s, uint64_t req_id, duwp_result *out)
{
    if (!s || !out) return DUWP_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return DUWP_ENOTFOUND;
    Request *r = it->second;
    if (!r->finished) return DUWP_PENDING;
    // a finished request is reported once, then released by the next poll of the same id
    if (r->slot == -2) {
        s->all.erase(it);
        delete r;
        return DUWP_ENOTFOUND;
    }
    std::memset(out, 0, sizeof *out);
    out->status = r->status;
    out->n_cells = static_cast<int32_t>(r->rho.size());
    out->steps = r->done_steps;
    out->particle_updates = r->updates0;
    out->queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
    out->run_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_admit).count();
    out->step_p50_ms = percentile(r->step_ms, 0.5);
    out->step_p99_ms = percentile(r->step_ms, 0.99);
    out->rho = r->rho.data();
    out->u = r->u.data();
    out->T = r->T.data();
    r->slot = -2;
    return DUWP_OK;
}

int duwp_server_destroy(duwp_server *s)
{
    if (!s) return DUWP_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    for (Lane *L : s->lanes)
        if (L->worker.joinable()) L->worker.join();
    for (Lane *L : s->lanes) delete L;
    for (auto &kv : s->all) delete kv.second;
    delete s;
    return DUWP_OK;
}

}  // extern "C"

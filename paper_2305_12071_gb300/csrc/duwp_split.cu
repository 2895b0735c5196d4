// duwp_split.cu -- one DUWP instance split into contiguous cell ranges, each range a part with its
// own engine (on one GPU or one GPU per part), stepped in lockstep with an exchange between parts.
//
// The method itself is per cell (Sec. 3.4: absorption, re-sampling and collisions act on a cell's
// own list; the transport moves particles between cells; the update of a cell reads the wave flux at
// its two faces), so a part needs from its neighbours, every step:
//   - after the transport, the particles that crossed into its cells: the run of the neighbour's
//     edge cell moving one cell across the boundary (with its exact moment sums, Eq. fp), written
//     into the part's phantom cell where its own edge cell expects the neighbouring run, and the
//     farther movers, merged into its far-mover list with their global sort keys (new cell, source
//     cell, position in the source list) before that list is sorted;
//   - after the cell update, the state of the neighbouring edge cell (a one-cell halo), copied into
//     the phantom cell, from which the wave flux of the boundary face and the NS-corrected sampling
//     read it.
// Every cell then sees the same list in the same order, the same generator ids (global cell
// indices) and the same sums as in the undivided run, so a split run equals it bit for bit.  The
// exchange goes through the host and plain device copies (peer copies across GPUs): no kernel of one
// part waits on another.
#include <cstring>
#include <new>
#include <vector>

#include "duwp_engine.h"
#include "duwp_launch.h"

using namespace duwp;

struct duwp_split {
    int32_t C = 0;                       // cells of the whole domain
    int fp32 = 1;
    std::vector<duwp_handle *> part;
    std::vector<int32_t> c0, c1;
    std::vector<int> device;
    int64_t steps = 0;
};

namespace {

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int d)
    {
        cudaGetDevice(&prev);
        if (d != prev) cudaSetDevice(d);
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define SPLIT_CU(call)                              \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) {                    \
            set_cuda_error(e_, #call);              \
            return DUWP_ECUDA;                      \
        }                                           \
    } while (0)

template <typename T>
int read_dev(int dev, T *host, const T *src, size_t n)
{
    DeviceScope d(dev);
    if (n) SPLIT_CU(cudaMemcpy(host, src, sizeof(T) * n, cudaMemcpyDeviceToHost));
    return DUWP_OK;
}

template <typename T>
int write_dev(int dev, T *dst, const T *host, size_t n)
{
    DeviceScope d(dev);
    if (n) SPLIT_CU(cudaMemcpy(dst, host, sizeof(T) * n, cudaMemcpyHostToDevice));
    return DUWP_OK;
}

// What one part hands to its neighbours after the transport.
struct EdgeRuns {
    int32_t nL = 0, nR = 0;              // L run of the first cell, R run of the last cell
    int64_t La = 0, Rend = 0;            // where they lie in the write buffer
    int64_t AL[4] = {0, 0, 0, 0}, AR[4] = {0, 0, 0, 0};
    std::vector<unsigned char> far;      // the unsorted far-mover list (FarItem records)
    int32_t nfar = 0;
};

int sync_part(duwp_split *s, int r)
{
    DeviceScope d(s->device[r]);
    SPLIT_CU(cudaStreamSynchronize(s->part[r]->eng.stream));
    int32_t err = 0;
    SPLIT_CU(cudaMemcpy(&err, s->part[r]->eng.dev.err, sizeof err, cudaMemcpyDeviceToHost));
    return err ? err : DUWP_OK;
}

int collect(duwp_split *s, int r, int wp, EdgeRuns &o, size_t item)
{
    Engine &E = s->part[r]->eng;
    const int dv = s->device[r];
    const int g0 = E.inst[0].cell_base + 1, g1 = g0 + s->c1[r] - s->c0[r] - 1;   // first, last cell
    int rc;
    int32_t sb0 = 0, sb1 = 0;
    int64_t off0 = 0, off1 = 0;
    if ((rc = read_dev(dv, &o.nL, E.dev.nL[wp] + g0, 1)) || (rc = read_dev(dv, &o.nR, E.dev.nR[wp] + g1, 1)) ||
        (rc = read_dev(dv, &sb0, E.dev.slotsb[wp] + g0, 1)) || (rc = read_dev(dv, &sb1, E.dev.slotsb[wp] + g1, 1)) ||
        (rc = read_dev(dv, &off0, E.dev.off[wp] + g0, 1)) || (rc = read_dev(dv, &off1, E.dev.off[wp] + g1, 1)) ||
        (rc = read_dev(dv, o.AL, E.dev.AL + 4 * static_cast<size_t>(g0), 4)) ||
        (rc = read_dev(dv, o.AR, E.dev.AR + 4 * static_cast<size_t>(g1), 4)) ||
        (rc = read_dev(dv, &o.nfar, E.dev.far_count, 1)))
        return rc;
    o.La = off0 + sb0;
    o.Rend = off1 + 2 * static_cast<int64_t>(sb1);
    if (o.nfar > E.far_cap) return DUWP_EOVERFLOW;
    o.far.resize(static_cast<size_t>(o.nfar) * item);
    return read_dev(dv, o.far.data(), static_cast<const unsigned char *>(E.dev.far_app), o.far.size());
}

// The run of cnt records at src of part a copied to dst of part b.
int copy_records(duwp_split *s, int b, void *dst, int a, const void *src, size_t bytes)
{
    if (!bytes) return DUWP_OK;
    DeviceScope d(s->device[b]);
    if (s->device[a] == s->device[b]) SPLIT_CU(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToDevice));
    else SPLIT_CU(cudaMemcpyPeer(dst, s->device[b], src, s->device[a], bytes));
    return DUWP_OK;
}

// Exchange after the transport of a step whose write parity is wp.
int exchange_particles(duwp_split *s, int wp)
{
    const int R = static_cast<int>(s->part.size());
    const size_t item = s->fp32 ? sizeof(FarItem<RecF>) : sizeof(FarItem<RecD>);
    const size_t rec = s->fp32 ? sizeof(RecF) : sizeof(RecD);
    std::vector<EdgeRuns> ed(static_cast<size_t>(R));
    for (int r = 0; r < R; ++r) {
        int rc = sync_part(s, r);
        if (rc) return rc;
        if ((rc = collect(s, r, wp, ed[r], item))) return rc;
    }
    for (int r = 0; r < R; ++r) {
        Engine &E = s->part[r]->eng;
        const int dv = s->device[r];
        const int base = E.inst[0].cell_base;
        const int gl = base, gr = base + 1 + (s->c1[r] - s->c0[r]);   // left and right phantom cells
        unsigned char *buf = static_cast<unsigned char *>(E.dev.buf[wp]);
        int rc;
        if (r > 0) {
            // the left neighbour's last cell moving right: its R run (stored backwards from Rend)
            const EdgeRuns &n = ed[r - 1];
            if (n.nR > E.pcap) return DUWP_EOVERFLOW;
            const int64_t off = E.capacity, sb = E.pcap / 2;        // Rend here = capacity + pcap
            const Engine &N = s->part[r - 1]->eng;
            const unsigned char *src = static_cast<const unsigned char *>(N.dev.buf[wp]) + rec * static_cast<size_t>(n.Rend - n.nR);
            if ((rc = copy_records(s, r, buf + rec * static_cast<size_t>(off + 2 * sb - n.nR), r - 1, src, rec * static_cast<size_t>(n.nR))))
                return rc;
            const int32_t sbi = static_cast<int32_t>(sb);
            if ((rc = write_dev(dv, E.dev.off[wp] + gl, &off, 1)) || (rc = write_dev(dv, E.dev.slotsb[wp] + gl, &sbi, 1)) ||
                (rc = write_dev(dv, E.dev.nR[wp] + gl, &n.nR, 1)) || (rc = write_dev(dv, E.dev.AR + 4 * static_cast<size_t>(gl), n.AR, 4)))
                return rc;
        }
        if (r + 1 < R) {
            // the right neighbour's first cell moving left: its L run (forward from La)
            const EdgeRuns &n = ed[r + 1];
            if (n.nL > E.pcap) return DUWP_EOVERFLOW;
            const int64_t off = E.capacity + E.pcap;
            const int32_t sb = 0;
            const Engine &N = s->part[r + 1]->eng;
            const unsigned char *src = static_cast<const unsigned char *>(N.dev.buf[wp]) + rec * static_cast<size_t>(n.La);
            if ((rc = copy_records(s, r, buf + rec * static_cast<size_t>(off), r + 1, src, rec * static_cast<size_t>(n.nL))))
                return rc;
            if ((rc = write_dev(dv, E.dev.off[wp] + gr, &off, 1)) || (rc = write_dev(dv, E.dev.slotsb[wp] + gr, &sb, 1)) ||
                (rc = write_dev(dv, E.dev.nL[wp] + gr, &n.nL, 1)) || (rc = write_dev(dv, E.dev.AL + 4 * static_cast<size_t>(gr), n.AL, 4)))
                return rc;
        }
        // far movers of the other parts whose new cell is one of this part's cells, with their keys
        // taken to this part's cell numbering (global cell g -> base + 1 + g - c0)
        std::vector<unsigned char> in;
        for (int q = 0; q < R; ++q) {
            if (q == r) continue;
            const int qbase = s->part[q]->eng.inst[0].cell_base;
            for (int32_t k = 0; k < ed[q].nfar; ++k) {
                int32_t key[3];
                std::memcpy(key, ed[q].far.data() + item * static_cast<size_t>(k), sizeof key);
                const int32_t gdest = s->c0[q] + (key[0] - qbase - 1), gsrc = s->c0[q] + (key[1] - qbase - 1);
                if (gdest < s->c0[r] || gdest >= s->c1[r]) continue;
                const size_t at = in.size();
                in.resize(at + item);
                std::memcpy(in.data() + at, ed[q].far.data() + item * static_cast<size_t>(k), item);
                const int32_t nk[2] = {base + 1 + (gdest - s->c0[r]), base + 1 + (gsrc - s->c0[r])};
                std::memcpy(in.data() + at, nk, sizeof nk);
            }
        }
        if (!in.empty()) {
            const int32_t n_in = static_cast<int32_t>(in.size() / item);
            if (ed[r].nfar + n_in > E.far_cap) return DUWP_EOVERFLOW;
            const int32_t total = ed[r].nfar + n_in;
            if ((rc = write_dev(dv, static_cast<unsigned char *>(E.dev.far_app) + item * static_cast<size_t>(ed[r].nfar), in.data(), in.size())) ||
                (rc = write_dev(dv, E.dev.far_count, &total, 1)))
                return rc;
        }
    }
    return DUWP_OK;
}

// The one-cell halo: the state of each neighbouring edge cell into the phantom cell.
int exchange_halo(duwp_split *s)
{
    const int R = static_cast<int>(s->part.size());
    for (int r = 0; r < R; ++r) {
        const int rc = sync_part(s, r);
        if (rc) return rc;
    }
    for (int r = 0; r < R; ++r) {
        Engine &E = s->part[r]->eng;
        const int base = E.inst[0].cell_base;
        for (int side = 0; side < 2; ++side) {
            const int q = side ? r + 1 : r - 1;
            if (q < 0 || q >= R) continue;
            const Engine &N = s->part[q]->eng;
            const int nbase = N.inst[0].cell_base;
            const int g_src = side ? nbase + 1 : nbase + (s->c1[q] - s->c0[q]);   // its first / last cell
            const int g_dst = side ? base + 1 + (s->c1[r] - s->c0[r]) : base;     // my right / left phantom
            double prim[5];
            int32_t valid = 0;
            int rc;
            if ((rc = read_dev(s->device[q], prim, N.dev.prim + 5 * static_cast<size_t>(g_src), 5)) ||
                (rc = read_dev(s->device[q], &valid, N.dev.valid + g_src, 1)) ||
                (rc = write_dev(s->device[r], E.dev.prim + 5 * static_cast<size_t>(g_dst), prim, 5)) ||
                (rc = write_dev(s->device[r], E.dev.valid + g_dst, &valid, 1)))
                return rc;
        }
    }
    return DUWP_OK;
}

int enqueue_all(duwp_split *s, int ph)
{
    for (size_t r = 0; r < s->part.size(); ++r) {
        DeviceScope d(s->device[r]);
        const int rc = s->part[r]->eng.enqueue_phase(ph);
        if (rc) return rc;
    }
    return DUWP_OK;
}

}  // namespace

extern "C" int duwp_split_create(const duwp_params *p, int32_t parts, const int32_t *devices, duwp_alloc_fn alloc,
                                 duwp_free_fn free_fn, void *alloc_ctx, duwp_split **out)
{
    if (!p || !out || parts < 1 || parts > p->n_cells) return DUWP_EINVAL;
    *out = nullptr;
    duwp_split *s = new (std::nothrow) duwp_split;
    if (!s) return DUWP_ENOMEM;
    s->C = p->n_cells;
    s->fp32 = (p->precision == DUWP_FP32) ? 1 : 0;
    int cur = 0;
    cudaGetDevice(&cur);
    for (int32_t r = 0; r < parts; ++r) {
        const int32_t a = static_cast<int32_t>((static_cast<int64_t>(p->n_cells) * r) / parts);
        const int32_t b = static_cast<int32_t>((static_cast<int64_t>(p->n_cells) * (r + 1)) / parts);
        const int dv = devices ? devices[r] : cur;
        duwp_handle *h = new (std::nothrow) duwp_handle;
        if (!h) {
            duwp_split_destroy(s);
            return DUWP_ENOMEM;
        }
        int rc;
        {
            DeviceScope d(dv);
            h->eng.part_c0 = a;
            h->eng.part_c1 = b;
            rc = h->eng.create(p, 1, 0, 0, 0, nullptr, alloc, free_fn, alloc_ctx);
        }
        s->part.push_back(h);
        s->c0.push_back(a);
        s->c1.push_back(b);
        s->device.push_back(dv);
        if (rc != DUWP_OK) {
            duwp_split_destroy(s);
            return rc;
        }
    }
    // the first flux and plans with the neighbours' states in the phantom cells
    int rc = exchange_halo(s);
    for (int32_t r = 0; r < parts && rc == DUWP_OK; ++r) {
        DeviceScope d(s->device[r]);
        rc = s->part[r]->eng.enqueue_prepare();
    }
    for (int32_t r = 0; r < parts && rc == DUWP_OK; ++r) rc = sync_part(s, r);
    if (rc != DUWP_OK) {
        duwp_split_destroy(s);
        return rc;
    }
    *out = s;
    return DUWP_OK;
}

extern "C" int duwp_split_step(duwp_split *s, int32_t n_steps)
{
    if (!s || n_steps < 0) return DUWP_EINVAL;
    for (int32_t k = 0; k < n_steps; ++k) {
        const int wp = 1 - s->part[0]->eng.parity;
        int rc = enqueue_all(s, 1);
        if (!rc) rc = exchange_particles(s, wp);
        if (!rc) rc = enqueue_all(s, 2);
        if (!rc) rc = exchange_halo(s);
        if (!rc) rc = enqueue_all(s, 3);
        if (rc) return rc;
        for (auto *h : s->part) h->eng.steps_done += 1;
        s->steps += 1;
    }
    for (size_t r = 0; r < s->part.size(); ++r) {
        const int rc = sync_part(s, static_cast<int>(r));
        if (rc) return rc;
    }
    return DUWP_OK;
}

extern "C" int duwp_split_part(duwp_split *s, int32_t r, duwp_handle **h, int32_t *c0, int32_t *c1)
{
    if (!s || r < 0 || r >= static_cast<int32_t>(s->part.size())) return DUWP_EINVAL;
    if (h) *h = s->part[r];
    if (c0) *c0 = s->c0[r];
    if (c1) *c1 = s->c1[r];
    return DUWP_OK;
}

extern "C" int duwp_split_destroy(duwp_split *s)
{
    if (!s) return DUWP_EINVAL;
    for (size_t r = 0; r < s->part.size(); ++r) {
        DeviceScope d(s->device[r]);
        delete s->part[r];
    }
    delete s;
    return DUWP_OK;
}

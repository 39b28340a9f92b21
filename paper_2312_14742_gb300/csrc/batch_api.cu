// C ABI of batches: admission by device footprint, table upload, graph
// capture and replay of the batched step, per-box reductions and state export.
//
// Host-side bookkeeping mirrors what the device tables hold: the live list,
// the first work item of each live box, and each box's step count (which
// also gives the copy holding its current state, since the copies swap every
// step). Table edits are queued on the batch's stream from pinned staging
// buffers, so they take effect between the steps queued before and after them.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batch.h"
#include "host.h"
#include "lbm_tau1.h"

using namespace lbm;

namespace {

constexpr int RING = 64;  // pinned staging buffers in flight

struct Stage {
    void* p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
};

struct Slot {
    bool live = false;
    lbm_tau1_config cfg{};
    int64_t n = 0;
    void* buf[2] = {};
    uint8_t* flags = nullptr;
    uint64_t bytes = 0;
    int64_t steps = 0;
    int ntiles = 0;  // tiles per plane
    int tma = 0;     // stepped by the staged instance (table 1), else table 0
};

uint64_t round256(uint64_t b) { return (b + 255) & ~(uint64_t)255; }

}  // namespace

struct lbm_tau1_batch {
    lbm_tau1_batch_config cfg{};
    cudaStream_t stream = nullptr;   // the caller's stream: all steps and table edits
    cudaStream_t side = nullptr;     // admission uploads (mask copy, flags, state init)
    cudaStream_t capture = nullptr;  // private stream for graph capture
    cudaStream_t capture2 = nullptr; // second capture branch: the other table's chain
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaEvent_t side_done = nullptr;
    std::vector<Slot> slots;
    // two work tables: [0] boxes stepped by the register instance, [1] by the
    // staged (TMA) instance; both index the same box records
    BatchTable* dtable[2] = {};
    BatchDomain* ddom = nullptr;
    int* dlive[2] = {};
    int* dbegin[2] = {};
    bool nonempty[2] = {};
    CUtensorMap* dmaps = nullptr;  // [capacity][2]
    Stage ring[RING];
    int ring_pos = 0;
    int grid[2] = {}, tile_h = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t budget = 0, used = 0;
    double* red_partials = nullptr;
    double* red_out = nullptr;   // device [capacity][RED_FIELDS]
    double* red_host = nullptr;  // pinned copy
    unsigned int* dtimeouts = nullptr;  // device counter of staged-copy waits that ran out
    // queued statistics (stats_queue / stats_wait): their own device and
    // pinned buffers ([capacity][RED_FIELDS], then the timeout count), the
    // event after the copy, and what the host needs to finish them
    double* qred_out = nullptr;
    double* qred_host = nullptr;
    cudaEvent_t qev = nullptr;
    bool qpending = false;
    std::vector<int64_t> qn, qsteps;
    std::vector<lbm_tau1_config> qcfg;
    int nlive = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

lbm_status bfail(lbm_tau1_batch* b, lbm_status st, const std::string& msg)
{
    if (b) b->err = msg;
    else set_create_error(msg);
    return st;
}

// Staged-copy waits that ran out since the last call (the caller has
// synchronised the batch's stream); clears the counter.
unsigned int take_timeouts(lbm_tau1_batch* b)
{
    unsigned int v = 0;
    if (!b->dtimeouts) return 0;
    if (cudaMemcpy(&v, b->dtimeouts, sizeof(v), cudaMemcpyDefault) != cudaSuccess) return 0;
    if (v) cudaMemset(b->dtimeouts, 0, sizeof(v));
    return v;
}

lbm_status bcuda(lbm_tau1_batch* b, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, m);
}

#define BCUDA(b, call, what)                                 \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return bcuda(b, e_, what);    \
    } while (0)

// A pinned staging buffer of at least `bytes`; its previous copies are complete.
cudaError_t stage_get(lbm_tau1_batch* b, size_t bytes, Stage** out)
{
    Stage& s = b->ring[b->ring_pos];
    b->ring_pos = (b->ring_pos + 1) % RING;
    cudaError_t e = cudaSuccess;
    if (s.pending) {
        if ((e = cudaEventSynchronize(s.ev)) != cudaSuccess) return e;
        s.pending = false;
    }
    if (s.cap < bytes) {
        if (s.p) cudaFreeHost(s.p);
        s.p = nullptr;
        s.cap = 0;
        if ((e = cudaMallocHost(&s.p, bytes)) != cudaSuccess) return e;
        s.cap = bytes;
    }
    if (!s.ev && (e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    *out = &s;
    return cudaSuccess;
}

cudaError_t stage_done(Stage* s, cudaStream_t stream)
{
    cudaError_t e = cudaEventRecord(s->ev, stream);
    s->pending = e == cudaSuccess;
    return e;
}

// Work items of a box for a chunk height.
int box_items(const Slot& s, int chunk) { return s.ntiles * ((s.cfg.nz + chunk - 1) / chunk); }

// Rebuilds the live lists and item offsets of both tables and queues their
// upload. A table's chunk is the tallest of 32, 16, 8 planes that still gives
// at least two items per block of its persistent grid, else 4. A change in
// which tables are empty drops the captured graph (it launches only the
// non-empty ones).
lbm_status upload_table(lbm_tau1_batch* b)
{
    int nlive = 0;
    for (int t = 0; t < 2; ++t) {
        int chunk = 32;
        for (; chunk > 4; chunk /= 2) {
            int64_t tot = 0;
            for (const Slot& s : b->slots)
                if (s.live && s.tma == t) tot += box_items(s, chunk);
            if (tot >= 2 * (int64_t)b->grid[t]) break;
        }
        std::vector<int> live, begin;
        int items = 0;
        for (int i = 0; i < (int)b->slots.size(); ++i)
            if (b->slots[i].live && b->slots[i].tma == t) {
                live.push_back(i);
                begin.push_back(items);
                items += box_items(b->slots[i], chunk);
            }
        const int nd = (int)live.size();
        BatchTable hdr{};
        hdr.nitems = items;
        hdr.ndom = nd;
        hdr.done = 0;
        hdr.next = 0;
        hdr.chunk = chunk;
        hdr.live = b->dlive[t];
        hdr.item_begin = b->dbegin[t];
        hdr.dom = b->ddom;
        hdr.maps = b->dmaps;
        const size_t lb = (size_t)nd * sizeof(int);
        Stage* st = nullptr;
        BCUDA(b, stage_get(b, sizeof(hdr) + 2 * lb + 16, &st), "batch: staging buffer");
        unsigned char* p = static_cast<unsigned char*>(st->p);
        std::memcpy(p, &hdr, sizeof(hdr));
        if (nd) {
            std::memcpy(p + sizeof(hdr), live.data(), lb);
            std::memcpy(p + sizeof(hdr) + lb, begin.data(), lb);
            BCUDA(b, cudaMemcpyAsync(b->dlive[t], p + sizeof(hdr), lb, cudaMemcpyHostToDevice, b->stream),
                  "batch: table copy");
            BCUDA(b, cudaMemcpyAsync(b->dbegin[t], p + sizeof(hdr) + lb, lb, cudaMemcpyHostToDevice, b->stream),
                  "batch: table copy");
        }
        BCUDA(b, cudaMemcpyAsync(b->dtable[t], p, sizeof(hdr), cudaMemcpyHostToDevice, b->stream),
              "batch: table copy");
        BCUDA(b, stage_done(st, b->stream), "batch: staging event");
        if ((nd > 0) != b->nonempty[t] && b->gexec) {
            // the graph's launches follow which tables are non-empty
            BCUDA(b, cudaStreamSynchronize(b->stream), "batch: sync before graph rebuild");
            cudaGraphExecDestroy(b->gexec);
            cudaGraphDestroy(b->graph);
            b->gexec = nullptr;
            b->graph = nullptr;
        }
        b->nonempty[t] = nd > 0;
        nlive += nd;
    }
    b->nlive = nlive;
    return LBM_OK;
}

// One step of every live box: one launch per non-empty table.
cudaError_t launch_step_tables(lbm_tau1_batch* b, cudaStream_t s)
{
    for (int t = 1; t >= 0; --t)
        if (b->nonempty[t]) {
            cudaError_t e = launch_tau1_batch(b->cfg.q, b->cfg.storage, b->cfg.variant, t == 1, b->dtable[t],
                                              b->grid[t], s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

int launches_per_step(const lbm_tau1_batch* b) { return (b->nonempty[0] ? 1 : 0) + (b->nonempty[1] ? 1 : 0); }

lbm_status capture_graph(lbm_tau1_batch* b)
{
    const int k = b->cfg.graph_steps;
    BCUDA(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "batch: begin capture");
    cudaError_t le = cudaSuccess;
    if (b->nonempty[0] && b->nonempty[1]) {
        // the two tables hold different boxes: two independent chains of k
        // steps, which the GPU runs side by side (one fills the other's tails)
        le = cudaEventRecord(b->fork_ev, b->capture);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(b->capture2, b->fork_ev, 0);
        for (int t = 1; t >= 0; --t) {
            cudaStream_t cs = t == 1 ? b->capture : b->capture2;
            for (int i = 0; i < k && le == cudaSuccess; ++i)
                le = launch_tau1_batch(b->cfg.q, b->cfg.storage, b->cfg.variant, t == 1, b->dtable[t], b->grid[t], cs);
        }
        if (le == cudaSuccess) le = cudaEventRecord(b->join_ev, b->capture2);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(b->capture, b->join_ev, 0);
    } else {
        for (int i = 0; i < k && le == cudaSuccess; ++i) le = launch_step_tables(b, b->capture);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->capture, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, le != cudaSuccess ? le : ee, "batch: graph capture");
    }
    cudaGraphExec_t x = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&x, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        return bcuda(b, ie, "batch: graph instantiate");
    }
    b->graph = g;
    b->gexec = x;
    return LBM_OK;
}

void free_batch(lbm_tau1_batch* b)
{
    if (b->stream || b->side) {
        cudaStreamSynchronize(b->stream);
        if (b->side) cudaStreamSynchronize(b->side);
    }
    for (Slot& s : b->slots) {
        if (s.buf[0]) cudaFree(s.buf[0]);
        if (s.buf[1]) cudaFree(s.buf[1]);
        if (s.flags) cudaFree(s.flags);
    }
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (Stage& s : b->ring) {
        if (s.ev) { cudaEventSynchronize(s.ev); cudaEventDestroy(s.ev); }
        if (s.p) cudaFreeHost(s.p);
    }
    for (int t = 0; t < 2; ++t) {
        if (b->dtable[t]) cudaFree(b->dtable[t]);
        if (b->dlive[t]) cudaFree(b->dlive[t]);
        if (b->dbegin[t]) cudaFree(b->dbegin[t]);
    }
    if (b->ddom) cudaFree(b->ddom);
    if (b->dmaps) cudaFree(b->dmaps);
    if (b->red_partials) cudaFree(b->red_partials);
    if (b->red_out) cudaFree(b->red_out);
    if (b->red_host) cudaFreeHost(b->red_host);
    if (b->qred_out) cudaFree(b->qred_out);
    if (b->qred_host) cudaFreeHost(b->qred_host);
    if (b->qev) cudaEventDestroy(b->qev);
    if (b->dtimeouts) cudaFree(b->dtimeouts);
    if (b->side_done) cudaEventDestroy(b->side_done);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->capture2) cudaStreamDestroy(b->capture2);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->join_ev) cudaEventDestroy(b->join_ev);
}

lbm_status live_slot(lbm_tau1_batch* b, int32_t slot, const char* what)
{
    if (slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[slot].live)
        return bfail(b, LBM_EINVAL, std::string(what) + ": slot is not live");
    return LBM_OK;
}

bool sixteen_bit(int storage) { return storage == LBM_F16S || storage == LBM_BF16S; }

// Device address of the inverse scales of a box's current copy (16-bit), else NULL.
const float* dinv_of(lbm_tau1_batch* b, int32_t slot)
{
    if (!sixteen_bit(b->cfg.storage)) return nullptr;
    const int c = (int)(b->slots[slot].steps & 1);
    return &b->ddom[slot].scale[c][4];
}

}  // namespace

extern "C" {

uint64_t lbm_tau1_batch_footprint(int32_t storage, int32_t nx, int32_t ny, int32_t nz)
{
    if (storage < LBM_F64 || storage > LBM_BF16S || nx < 1 || ny < 1 || nz < 1) return 0;
    const uint64_t n = (uint64_t)nx * (uint64_t)ny * (uint64_t)nz;
    return 2 * round256(n * (uint64_t)node_bytes(storage)) + round256(n);
}

lbm_status lbm_tau1_batch_create(const lbm_tau1_batch_config* cfg, lbm_tau1_batch** out)
{
    if (out) *out = nullptr;
    if (!cfg || !out) return bfail(nullptr, LBM_EINVAL, "batch_create: NULL argument");
    if (cfg->q != 19 && cfg->q != 27) return bfail(nullptr, LBM_EINVAL, "batch_create: q must be 19 or 27");
    if (cfg->storage < LBM_F64 || cfg->storage > LBM_BF16S) return bfail(nullptr, LBM_EINVAL, "batch_create: bad storage");
    if (cfg->variant < 0 || cfg->variant >= tau1_tile_shapes(cfg->storage))
        return bfail(nullptr, LBM_EINVAL, "batch_create: bad variant");
    if (cfg->capacity < 1 || cfg->capacity > (1 << 20)) return bfail(nullptr, LBM_EINVAL, "batch_create: bad capacity");
    if (cfg->graph_steps < 0 || cfg->graph_steps > 100000)
        return bfail(nullptr, LBM_EINVAL, "batch_create: bad graph_steps");

    lbm_tau1_batch* b = new (std::nothrow) lbm_tau1_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "batch_create: host allocation failed");
    b->cfg = *cfg;
    if (b->cfg.graph_steps == 0) b->cfg.graph_steps = 100;
    b->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    b->slots.resize((size_t)cfg->capacity);
    const int cap = cfg->capacity;
    cudaError_t e = batch_prepare(cfg->q, cfg->storage, cfg->variant, false, &b->grid[0], &b->tile_h);
    if (e == cudaSuccess) e = batch_prepare(cfg->q, cfg->storage, cfg->variant, true, &b->grid[1], &b->tile_h);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side_done, cudaEventDisableTiming);
    for (int t = 0; t < 2; ++t) {
        if (e == cudaSuccess) e = cudaMalloc(&b->dtable[t], sizeof(BatchTable));
        if (e == cudaSuccess) e = cudaMalloc(&b->dlive[t], (size_t)cap * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&b->dbegin[t], (size_t)cap * sizeof(int));
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->ddom, (size_t)cap * sizeof(BatchDomain));
    if (e == cudaSuccess) e = cudaMalloc(&b->dmaps, (size_t)cap * 2 * sizeof(CUtensorMap));
    if (e == cudaSuccess) e = cudaMalloc(&b->red_partials, (size_t)1024 * RED_FIELDS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->red_out, (size_t)cap * RED_FIELDS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->dtimeouts, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->dtimeouts, 0, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&b->red_host, (size_t)cap * RED_FIELDS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->qred_out, ((size_t)cap * RED_FIELDS + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&b->qred_host, ((size_t)cap * RED_FIELDS + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->qev, cudaEventDisableTiming);
    if (e == cudaSuccess && cfg->hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        b->budget = (uint64_t)(0.9 * (double)fr);
    } else {
        b->budget = cfg->hbm_budget;
    }
    lbm_status st = LBM_OK;
    if (e != cudaSuccess) st = bcuda(nullptr, e, "batch_create: CUDA setup");
    if (st == LBM_OK) {
        st = upload_table(b);
        if (st != LBM_OK) set_create_error(b->err);
    }
    if (st == LBM_OK) {
        e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bcuda(nullptr, e, "batch_create: sync");
    }
    if (st != LBM_OK) {
        free_batch(b);
        delete b;
        return st;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_tau1_batch_admit(lbm_tau1_batch* b, const lbm_tau1_config* cfg, const uint8_t* solid, int on_device,
                                int32_t* slot)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_admit: NULL batch");
    if (slot) *slot = -1;
    if (!cfg || !solid || !slot) return bfail(b, LBM_EINVAL, "batch_admit: NULL argument");
    if (cfg->q != b->cfg.q || cfg->storage != b->cfg.storage)
        return bfail(b, LBM_EINVAL, "batch_admit: lattice and storage must match the batch");
    if (cfg->layout != LBM_DENSE || cfg->scheme != LBM_SCHEME_TAU1)
        return bfail(b, LBM_EINVAL, "batch_admit: boxes are dense-layout Tau1");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return bfail(b, LBM_EINVAL, "batch_admit: box sizes must be >= 1");
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(cfg->g[d])) return bfail(b, LBM_EINVAL, "batch_admit: g must be finite");
    const int64_t n = (int64_t)cfg->nx * cfg->ny * cfg->nz;
    if (!tau1_tiled_supported(cfg->q, cfg->storage, n)) return bfail(b, LBM_EINVAL, "batch_admit: box too large");
    const uint64_t need = lbm_tau1_batch_footprint(cfg->storage, cfg->nx, cfg->ny, cfg->nz);
    if (b->nlive >= b->cfg.capacity) return bfail(b, LBM_EBUSY, "batch_admit: capacity reached");
    if (need > b->budget - b->used) return bfail(b, LBM_EBUSY, "batch_admit: footprint exceeds the budget left");
    int id = -1;
    for (int i = 0; i < (int)b->slots.size(); ++i)
        if (!b->slots[i].live && !b->slots[i].buf[0]) { id = i; break; }
    if (id < 0) return bfail(b, LBM_EBUSY, "batch_admit: no free slot");
    Slot& s = b->slots[id];

    // device memory, geometry and initial state, on the side stream
    const size_t rb = (size_t)n * (size_t)node_bytes(cfg->storage);
    cudaError_t e = cudaMallocAsync(&s.buf[0], rb, b->side);
    if (e == cudaSuccess) e = cudaMallocAsync(&s.buf[1], rb, b->side);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&s.flags, (size_t)n, b->side);
    uint8_t* tmp = nullptr;
    const uint8_t* dsolid = solid;
    if (e == cudaSuccess && !on_device) {
        e = cudaMallocAsync((void**)&tmp, (size_t)n, b->side);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, solid, (size_t)n, cudaMemcpyDefault, b->side);
        dsolid = tmp;
    }
    int per[3] = {cfg->periodic[0] ? 1 : 0, cfg->periodic[1] ? 1 : 0, cfg->periodic[2] ? 1 : 0};
    if (e == cudaSuccess) e = launch_build_flags(cfg->q, cfg->nx, cfg->ny, cfg->nz, per, dsolid, s.flags, b->side);
    if (tmp) cudaFreeAsync(tmp, b->side);
    double gmax = 0;
    for (int d = 0; d < 3; ++d) gmax = std::fmax(gmax, std::fabs(cfg->g[d]));
    const double zero[4] = {0, 0, 0, 0};
    float sc[4];
    initial_scales(cfg->storage, zero, gmax, sc);
    for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = launch_import_state(cfg->storage, n, nullptr, s.buf[c], s.flags, sc, b->side);
    if (e == cudaSuccess) e = cudaEventRecord(b->side_done, b->side);
    if (e != cudaSuccess) {
        for (int c = 0; c < 2; ++c)
            if (s.buf[c]) { cudaFreeAsync(s.buf[c], b->side); s.buf[c] = nullptr; }
        if (s.flags) { cudaFreeAsync(s.flags, b->side); s.flags = nullptr; }
        return bcuda(b, e, "batch_admit: upload");
    }
    b->launches += 3;

    // the box's table record, after every queued step (the slot may have had an earlier box)
    BatchDomain rec{};
    rec.a.nx = cfg->nx;
    rec.a.ny = cfg->ny;
    rec.a.nz = cfg->nz;
    rec.a.timeouts = b->dtimeouts;
    for (int d = 0; d < 3; ++d) {
        rec.a.periodic[d] = per[d];
        rec.a.g[d] = cfg->g[d];
        rec.a.gf[d] = (float)cfg->g[d];
    }
    rec.buf[0] = s.buf[0];
    rec.buf[1] = s.buf[1];
    rec.ntx = (cfg->nx + 31) / 32;
    const int nty = (cfg->ny + b->tile_h - 1) / b->tile_h;
    rec.ntiles = rec.ntx * nty;
    rec.cur = 0;
    rec.step = 0;
    for (int c = 0; c < 2; ++c)
        for (int f = 0; f < 4; ++f) {
            rec.scale[c][f] = sc[f];
            rec.scale[c][4 + f] = 1.0f / sc[f];
        }
    rec.gfloor = (float)(64.0 * gmax);
    // staged tile columns for boxes of full tiles (16-bit rows start on 16 bytes only for even nx)
    CUtensorMap maps[2];
    rec.tma = cfg->nx % 32 == 0 && cfg->ny % b->tile_h == 0 &&
              !((cfg->storage == LBM_F16S || cfg->storage == LBM_BF16S) && cfg->nx % 2 != 0);
    for (int c = 0; c < 2 && rec.tma; ++c)
        if (encode_state_map(cfg->storage, s.buf[c], cfg->nx, cfg->ny, cfg->nz, b->tile_h + 2, &maps[c]) !=
            cudaSuccess)
            rec.tma = 0;
    Stage* st = nullptr;
    BCUDA(b, stage_get(b, sizeof(rec) + sizeof(maps), &st), "batch_admit: staging buffer");
    std::memcpy(st->p, maps, sizeof(maps));
    std::memcpy(static_cast<unsigned char*>(st->p) + sizeof(maps), &rec, sizeof(rec));
    BCUDA(b, cudaStreamWaitEvent(b->stream, b->side_done, 0), "batch_admit: wait");
    if (rec.tma)
        BCUDA(b, cudaMemcpyAsync(b->dmaps + 2 * id, st->p, sizeof(maps), cudaMemcpyHostToDevice, b->stream),
              "batch_admit: tensor map copy");
    BCUDA(b, cudaMemcpyAsync(b->ddom + id, static_cast<unsigned char*>(st->p) + sizeof(maps), sizeof(rec),
                             cudaMemcpyHostToDevice, b->stream),
          "batch_admit: record copy");
    BCUDA(b, stage_done(st, b->stream), "batch_admit: staging event");

    s.live = true;
    s.cfg = *cfg;
    s.n = n;
    s.bytes = need;
    s.steps = 0;
    s.ntiles = rec.ntiles;
    s.tma = rec.tma;
    b->used += need;
    if (lbm_status r = upload_table(b)) return r;
    *slot = id;
    return LBM_OK;
}

lbm_status lbm_tau1_batch_release(lbm_tau1_batch* b, int32_t slot)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_release: NULL batch");
    if (lbm_status st = live_slot(b, slot, "batch_release")) return st;
    Slot& s = b->slots[slot];
    s.live = false;
    if (lbm_status st = upload_table(b)) return st;
    // freed in stream order: after every queued step that reads them
    for (int c = 0; c < 2; ++c) {
        BCUDA(b, cudaFreeAsync(s.buf[c], b->stream), "batch_release: free");
        s.buf[c] = nullptr;
    }
    BCUDA(b, cudaFreeAsync(s.flags, b->stream), "batch_release: free");
    s.flags = nullptr;
    b->used -= s.bytes;
    s.bytes = 0;
    return LBM_OK;
}

lbm_status lbm_tau1_batch_step(lbm_tau1_batch* b, int64_t nsteps)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_step: NULL batch");
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "batch_step: nsteps < 0");
    if (b->nlive == 0 || nsteps == 0) return LBM_OK;
    const int64_t k = b->cfg.graph_steps;
    int64_t left = nsteps;
    if (left >= k && !b->gexec)
        if (lbm_status st = capture_graph(b)) return st;
    for (; left >= k; left -= k) {
        BCUDA(b, cudaGraphLaunch(b->gexec, b->stream), "batch_step: graph launch");
        b->launches += k * launches_per_step(b);
    }
    for (; left > 0; --left) {
        BCUDA(b, launch_step_tables(b, b->stream), "batch_step: launch");
        b->launches += launches_per_step(b);
    }
    for (Slot& s : b->slots)
        if (s.live) s.steps += nsteps;
    return LBM_OK;
}

lbm_status lbm_tau1_batch_stats(lbm_tau1_batch* b, int32_t n, const int32_t* slots, lbm_tau1_stats* out)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_stats: NULL batch");
    if (n < 0 || n > b->cfg.capacity || (n > 0 && (!slots || !out)))
        return bfail(b, LBM_EINVAL, "batch_stats: bad arguments");
    for (int i = 0; i < n; ++i)
        if (lbm_status st = live_slot(b, slots[i], "batch_stats")) return st;
    for (int i = 0; i < n; ++i) {
        const Slot& s = b->slots[slots[i]];
        const void* f[4] = {s.buf[s.steps & 1], nullptr, nullptr, nullptr};
        cudaError_t e = launch_reduce(b->cfg.storage, true, s.n, f, nullptr, s.flags, s.cfg.g, b->red_partials,
                                      b->red_out + (size_t)i * RED_FIELDS, b->stream, dinv_of(b, slots[i]));
        b->launches += 2;
        if (e != cudaSuccess) return bcuda(b, e, "batch_stats: kernel");
    }
    if (n == 0) return LBM_OK;
    BCUDA(b, cudaMemcpyAsync(b->red_host, b->red_out, (size_t)n * RED_FIELDS * sizeof(double), cudaMemcpyDefault,
                             b->stream), "batch_stats: copy");
    BCUDA(b, cudaStreamSynchronize(b->stream), "batch_stats: sync");
    if (unsigned t = take_timeouts(b))
        return bfail(b, LBM_ETIMEOUT, "batch_stats: " + std::to_string(t) + " staged-copy waits ran out");
    lbm_status worst = LBM_OK;
    for (int i = 0; i < n; ++i) {
        const Slot& s = b->slots[slots[i]];
        if (fill_stats(b->red_host + (size_t)i * RED_FIELDS, s.n, s.cfg.g, s.steps, &out[i]) != LBM_OK)
            worst = LBM_EDIVERGED;
    }
    if (worst != LBM_OK) return bfail(b, worst, "batch_stats: a box diverged (non-finite value or |u| > 0.3)");
    return LBM_OK;
}

lbm_status lbm_tau1_batch_selftest_timeout(lbm_tau1_batch* b)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_selftest_timeout: NULL batch");
    BCUDA(b, launch_selftest_timeout(b->dtimeouts, b->stream), "batch_selftest_timeout: launch");
    ++b->launches;
    return LBM_OK;
}

lbm_status lbm_tau1_batch_stats_queue(lbm_tau1_batch* b, int32_t n, const int32_t* slots)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_stats_queue: NULL batch");
    if (b->qpending) return bfail(b, LBM_ESTATE, "batch_stats_queue: the previous queued statistics were not taken");
    if (n < 0 || n > b->cfg.capacity || (n > 0 && !slots)) return bfail(b, LBM_EINVAL, "batch_stats_queue: bad arguments");
    for (int i = 0; i < n; ++i)
        if (lbm_status st = live_slot(b, slots[i], "batch_stats_queue")) return st;
    b->qn.assign((size_t)n, 0);
    b->qsteps.assign((size_t)n, 0);
    b->qcfg.assign((size_t)n, lbm_tau1_config{});
    for (int i = 0; i < n; ++i) {
        const Slot& s = b->slots[slots[i]];
        const void* f[4] = {s.buf[s.steps & 1], nullptr, nullptr, nullptr};
        cudaError_t e = launch_reduce(b->cfg.storage, true, s.n, f, nullptr, s.flags, s.cfg.g, b->red_partials,
                                      b->qred_out + (size_t)i * RED_FIELDS, b->stream, dinv_of(b, slots[i]));
        b->launches += 2;
        if (e != cudaSuccess) return bcuda(b, e, "batch_stats_queue: kernel");
        b->qn[(size_t)i] = s.n;
        b->qsteps[(size_t)i] = s.steps;
        b->qcfg[(size_t)i] = s.cfg;
    }
    // the statistics and the timeout count (as a double after them), then the count cleared
    const size_t tail = (size_t)n * RED_FIELDS;
    BCUDA(b, cudaMemcpyAsync(b->qred_host, b->qred_out, tail * sizeof(double), cudaMemcpyDefault, b->stream),
          "batch_stats_queue: copy");
    unsigned int* tcount = reinterpret_cast<unsigned int*>(b->qred_host + tail);
    BCUDA(b, cudaMemcpyAsync(tcount, b->dtimeouts, sizeof(unsigned int), cudaMemcpyDefault, b->stream),
          "batch_stats_queue: copy");
    BCUDA(b, cudaMemsetAsync(b->dtimeouts, 0, sizeof(unsigned int), b->stream), "batch_stats_queue: clear");
    BCUDA(b, cudaEventRecord(b->qev, b->stream), "batch_stats_queue: event");
    b->qpending = true;
    return LBM_OK;
}

lbm_status lbm_tau1_batch_stats_wait(lbm_tau1_batch* b, lbm_tau1_stats* out)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_stats_wait: NULL batch");
    if (!b->qpending) return bfail(b, LBM_ESTATE, "batch_stats_wait: no statistics queued");
    const int n = (int)b->qn.size();
    if (n > 0 && !out) return bfail(b, LBM_EINVAL, "batch_stats_wait: NULL output");
    b->qpending = false;
    BCUDA(b, cudaEventSynchronize(b->qev), "batch_stats_wait: sync");
    const unsigned int t = *reinterpret_cast<const unsigned int*>(b->qred_host + (size_t)n * RED_FIELDS);
    if (t) return bfail(b, LBM_ETIMEOUT, "batch_stats_wait: " + std::to_string(t) + " staged-copy waits ran out");
    lbm_status worst = LBM_OK;
    for (int i = 0; i < n; ++i)
        if (fill_stats(b->qred_host + (size_t)i * RED_FIELDS, b->qn[(size_t)i], b->qcfg[(size_t)i].g,
                       b->qsteps[(size_t)i], &out[i]) != LBM_OK)
            worst = LBM_EDIVERGED;
    if (worst != LBM_OK) return bfail(b, worst, "batch_stats_wait: a box diverged (non-finite value or |u| > 0.3)");
    return LBM_OK;
}

lbm_status lbm_tau1_batch_get_fields(lbm_tau1_batch* b, int32_t slot, double* drho, double* ux, double* uy,
                                     double* uz, int on_device)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_get_fields: NULL batch");
    if (lbm_status st = live_slot(b, slot, "batch_get_fields")) return st;
    const Slot& s = b->slots[slot];
    double* dst[4] = {drho, ux, uy, uz};
    const size_t bytes = (size_t)s.n * sizeof(double);
    double* tmp = nullptr;
    BCUDA(b, cudaMallocAsync((void**)&tmp, 4 * bytes, b->stream), "batch_get_fields: staging allocation");
    double* ddst[4];
    for (int f = 0; f < 4; ++f) ddst[f] = (on_device && dst[f]) ? dst[f] : tmp + f * s.n;
    cudaError_t e = launch_export_state(b->cfg.storage, s.n, s.buf[s.steps & 1], ddst, s.flags, nullptr, b->stream,
                                        dinv_of(b, slot));
    ++b->launches;
    if (e != cudaSuccess) { cudaFreeAsync(tmp, b->stream); return bcuda(b, e, "batch_get_fields: export kernel"); }
    if (!on_device)
        for (int f = 0; f < 4; ++f)
            if (dst[f]) {
                e = cudaMemcpyAsync(dst[f], ddst[f], bytes, cudaMemcpyDefault, b->stream);
                if (e != cudaSuccess) { cudaFreeAsync(tmp, b->stream); return bcuda(b, e, "batch_get_fields: copy"); }
            }
    cudaFreeAsync(tmp, b->stream);
    if (!on_device) BCUDA(b, cudaStreamSynchronize(b->stream), "batch_get_fields: sync");
    return LBM_OK;
}

lbm_status lbm_tau1_batch_synchronize(lbm_tau1_batch* b)
{
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch_synchronize: NULL batch");
    BCUDA(b, cudaStreamSynchronize(b->stream), "batch_synchronize");
    if (unsigned t = take_timeouts(b))
        return bfail(b, LBM_ETIMEOUT, "batch_synchronize: " + std::to_string(t) + " staged-copy waits ran out");
    return LBM_OK;
}

lbm_status lbm_tau1_batch_destroy(lbm_tau1_batch* b)
{
    if (!b) return LBM_OK;
    free_batch(b);
    delete b;
    return LBM_OK;
}

int32_t lbm_tau1_batch_live(const lbm_tau1_batch* b) { return b ? b->nlive : 0; }

uint64_t lbm_tau1_batch_bytes_free(const lbm_tau1_batch* b) { return b ? b->budget - b->used : 0; }

int64_t lbm_tau1_batch_launch_count(const lbm_tau1_batch* b) { return b ? b->launches : 0; }

const char* lbm_tau1_batch_last_error(const lbm_tau1_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"

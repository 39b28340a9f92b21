// C ABI of the Tau1 solver: handle life cycle, geometry, state I/O, stepping
// and reductions. Declarations and the contract of each entry point are in
// include/lbm_tau1.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "host.h"
#include "kernels.h"
#include "lbm_tau1.h"

using namespace lbm;

struct lbm_tau1 {
    lbm_tau1_config cfg{};
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    size_t node_bytes = 0;      // bytes per node record {drho, ux, uy, uz}
    void* buf[2] = {};          // ping-pong copies of the state records
    int cur = 0;                // buf[cur] is the current (pre) state
    void* fbuf[2] = {};         // BGK scheme: ping-pong populations [q][n]
    uint32_t* bgk_mask = nullptr;  // BGK scheme: wall links of every node
    int fcur = 0;
    bool bgk = false;
    uint8_t* flags = nullptr;   // node flags
    double* red_partials = nullptr;
    double* red_out = nullptr;  // device, RED_FIELDS doubles
    double* red_host = nullptr; // pinned host copy of red_out
    bool has_geometry = false;
    int64_t step = 0;
    int64_t n_fluid = -1;
    float scale[4] = {1, 1, 1, 1};      // host mirror of the 16-bit scales
    float inv_scale[4] = {1, 1, 1, 1};
    float* dscale = nullptr;            // 16-bit storage: device {S_f, 1/S_f}
    float* rescale_scratch = nullptr;   // 16-bit storage: maxima partials + ratios
    float scale_host[8] = {};           // staging for scale copies
    int kernel = LBM_KERNEL_SIMPLE;
    int variant = 0;            // tile-shape variant of the tiled kernel
    bool sparse = false;        // fluid-list layout: buf holds nf records
    int64_t nf = 0;             // sparse: fluid nodes in the list
    int* pos = nullptr;         // sparse: box node of each list entry
    int* nbr = nullptr;         // sparse: neighbour table [(q-1)][nf]
    int64_t launches = 0;
    unsigned int* dtimeouts = nullptr;  // device counter of staged-copy waits that ran out
    bool compact = false;       // compact layout: dense records, work split by tile column
    double cthr = 0.3;          // compact: fluid fraction from which a tile column is tiled
    bool c_tiled_ok = false;    // compact: the row-pair kernel takes the box's tile columns
    CompactTiles ctile{};       // compact: tile columns of the row-pair variant h->variant
    int ccounted = -1;          // compact: variant whose columns ccounts holds (-1: none)
    int64_t ccap = 0;           // compact: tile columns the three arrays below can hold
    int* ccounts = nullptr;     // compact: device fluid count of every tile column
    std::vector<int> ccounts_host;
    int* ctiles = nullptr;      // compact: tile columns of the row-pair kernel [columns]
    int* clisted = nullptr;     // compact: tile columns of the node list, then their offsets [2 columns]
    int* cnodes = nullptr;      // compact: the node list [fluid nodes]
    int64_t n_ctiles = 0, n_clisted = 0, n_cnodes = 0, c_tiled_fluid = 0, c_empty = 0;
    cudaStream_t cside = nullptr;   // compact: the node-list kernel's stream when both kernels run
    cudaEvent_t cfork = nullptr, cjoin = nullptr;
    int p_axis = -1;            // constant-density faces on this axis (-1: none)
    double p_lo = 1.0, p_hi = 1.0;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

lbm_status fail(lbm_tau1* h, lbm_status st, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return st;
}

lbm_status cuda_fail(lbm_tau1* h, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, m);
}

#define LBM_CUDA(h, call, what)                          \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

size_t storage_node_bytes(int st) { return (st >= LBM_F64 && st <= LBM_BF16S) ? (size_t)node_bytes(st) : 0; }

void free_all(lbm_tau1* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (int b = 0; b < 2; ++b) {
        if (h->buf[b]) cudaFree(h->buf[b]);
        if (h->fbuf[b]) cudaFree(h->fbuf[b]);
    }
    if (h->bgk_mask) cudaFree(h->bgk_mask);
    if (h->flags) cudaFree(h->flags);
    if (h->pos) cudaFree(h->pos);
    if (h->nbr) cudaFree(h->nbr);
    if (h->red_partials) cudaFree(h->red_partials);
    if (h->red_out) cudaFree(h->red_out);
    if (h->red_host) cudaFreeHost(h->red_host);
    if (h->dscale) cudaFree(h->dscale);
    if (h->rescale_scratch) cudaFree(h->rescale_scratch);
    if (h->dtimeouts) cudaFree(h->dtimeouts);
    if (h->ccounts) cudaFree(h->ccounts);
    if (h->ctiles) cudaFree(h->ctiles);
    if (h->clisted) cudaFree(h->clisted);
    if (h->cnodes) cudaFree(h->cnodes);
    if (h->cfork) cudaEventDestroy(h->cfork);
    if (h->cjoin) cudaEventDestroy(h->cjoin);
    if (h->cside) cudaStreamDestroy(h->cside);
}

// Staged-copy waits that ran out since the last call (reads the device
// counter on the handle's stream, then clears it).
unsigned int take_timeouts(lbm_tau1* h)
{
    unsigned int v = 0;
    if (!h->dtimeouts) return 0;
    if (cudaMemcpyAsync(&v, h->dtimeouts, sizeof(v), cudaMemcpyDefault, h->stream) != cudaSuccess) return 0;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return 0;
    if (v) cudaMemsetAsync(h->dtimeouts, 0, sizeof(v), h->stream);
    return v;
}

lbm_status check_ptr(lbm_tau1* h, const void* p, int on_device, const char* name)
{
    if (!p) return LBM_OK;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(h, LBM_EINVAL, std::string(name) + ": unknown pointer"); }
    const bool dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (on_device && !dev) return fail(h, LBM_EINVAL, std::string(name) + ": on_device=1 but not a device pointer");
    return LBM_OK;
}

void fill_args(const lbm_tau1* h, StepArgs& a)
{
    a.nx = h->cfg.nx;
    a.ny = h->cfg.ny;
    a.nz = h->cfg.nz;
    for (int d = 0; d < 3; ++d) {
        a.periodic[d] = h->cfg.periodic[d] ? 1 : 0;
        a.g[d] = h->cfg.g[d];
        a.gf[d] = (float)h->cfg.g[d];
    }
    a.pre = h->buf[h->cur];
    a.post = h->buf[h->cur ^ 1];
    a.dscale = h->dscale;
    a.seed = (uint32_t)(h->step + 1) * 0x9E3779B9u;
    a.timeouts = h->dtimeouts;
    for (int f = 0; f < 4; ++f) {
        a.inv_scale[f] = h->inv_scale[f];
        a.scale[f] = h->scale[f];
    }
}

int variant_count(const lbm_tau1* h)
{
    if (h->cfg.q == LBM_D2Q9) return 1;
    if (h->compact) return 2 * tau1_rowpair_shapes(h->cfg.storage);
    return (!h->bgk && h->kernel == LBM_KERNEL_TILED) ? tau1_tiled_variants(h->cfg.q, h->cfg.storage) : 1;
}

constexpr int64_t RESCALE_EVERY = 64;  // 16-bit storage: steps between scale checks

bool sixteen(const lbm_tau1* h) { return h->cfg.storage == LBM_F16S || h->cfg.storage == LBM_BF16S; }

lbm_status upload_scales(lbm_tau1* h)
{
    if (!h->dscale) return LBM_OK;
    for (int f = 0; f < 4; ++f) {
        h->scale_host[f] = h->scale[f];
        h->scale_host[4 + f] = h->inv_scale[f];
    }
    LBM_CUDA(h, cudaMemcpyAsync(h->dscale, h->scale_host, 8 * sizeof(float), cudaMemcpyDefault, h->stream),
             "scales upload");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "scales upload sync");
    return LBM_OK;
}

// The device scales may have changed while stepping: refresh the host mirror.
lbm_status download_scales(lbm_tau1* h)
{
    if (!h->dscale) return LBM_OK;
    LBM_CUDA(h, cudaMemcpyAsync(h->scale_host, h->dscale, 8 * sizeof(float), cudaMemcpyDefault, h->stream),
             "scales download");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "scales download sync");
    for (int f = 0; f < 4; ++f) {
        h->scale[f] = h->scale_host[f];
        h->inv_scale[f] = h->scale_host[4 + f];
    }
    return LBM_OK;
}

// Default 16-bit scales before any state is known: sized for velocities up
// to 100 |g| (the first rescale check corrects them).
double gmax_of(const lbm_tau1* h)
{
    double gmax = 0;
    for (int d = 0; d < 3; ++d) gmax = std::fmax(gmax, std::fabs(h->cfg.g[d]));
    return gmax;
}

// Scales of a state whose fields have maxima m (headroom rule, scale.cu).
void set_scales(lbm_tau1* h, const double m[4])
{
    initial_scales(h->cfg.storage, m, gmax_of(h), h->scale);
    for (int f = 0; f < 4; ++f) h->inv_scale[f] = 1.0f / h->scale[f];
}

// BGK: state records of the current step (before reading the state). The
// newest copy holds post-collision populations of step n; gathering from the
// previous copy yields the populations that arrived at step n, whose moments
// are the state Tau1 reports. At step 0 the imported state is current.
lbm_status bgk_refresh_state(lbm_tau1* h)
{
    if (!h->bgk || h->step == 0) return LBM_OK;
    StepArgs a;
    fill_args(h, a);
    cudaError_t e = launch_bgk_moments(h->cfg.q, h->cfg.storage, a, h->fbuf[h->fcur ^ 1], h->buf[h->cur],
                                       h->bgk_mask, h->stream);
    ++h->launches;
    if (e != cudaSuccess) return cuda_fail(h, e, "bgk moments kernel");
    return LBM_OK;
}

// BGK: wall links from the node flags, populations from the current state records.
lbm_status bgk_from_state(lbm_tau1* h)
{
    if (!h->bgk) return LBM_OK;
    StepArgs a;
    fill_args(h, a);
    {
        cudaError_t e = launch_bgk_mask(h->cfg.q, a, h->flags, h->bgk_mask, h->stream);
        ++h->launches;
        if (e != cudaSuccess) return cuda_fail(h, e, "bgk wall-link kernel");
    }
    // both copies: the step kernel writes fluid nodes only, so the solid
    // nodes of the other copy must already hold their NaN marker
    for (int b = 0; b < 2; ++b) {
        cudaError_t e = launch_bgk_init(h->cfg.q, h->cfg.storage, a, h->buf[h->cur], h->fbuf[b], h->stream);
        ++h->launches;
        if (e != cudaSuccess) return cuda_fail(h, e, "bgk init kernel");
    }
    return LBM_OK;
}

// Autotune cache key: device, lattice, storage, layout, size bucket
// (ceil log2 of the node count) and whether every tile is full (the staged
// kernel's condition), e.g. "NVIDIA GB300/D3Q19/F32/dense/n2^24/full".
std::string tune_key(const lbm_tau1* h)
{
    int dev = 0;
    cudaDeviceProp p{};
    std::string name = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess) name = p.name;
    static const char* st[] = {"F64", "F32", "F16S", "BF16S"};
    int lg = 0;
    while (((int64_t)1 << lg) < h->n) ++lg;
    const bool full = h->cfg.nx % 32 == 0 && h->cfg.ny % 16 == 0;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s/D3Q%d/%s/%s/n2^%d/%s", name.c_str(), h->cfg.q, st[h->cfg.storage],
                  h->sparse ? "sparse" : "dense", lg, full ? "full" : "ragged");
    return buf;
}

// Sparse layout: numbers the fluid nodes (prefix sum of the flags), then
// allocates and fills the list records' copies, pos and the neighbour table.
lbm_status build_fluid_list(lbm_tau1* h)
{
    const int nb = sparse_scan_blocks(h->n);
    int* counts = nullptr;
    int* idx = nullptr;
    LBM_CUDA(h, cudaMallocAsync((void**)&counts, (size_t)(nb + 1) * sizeof(int), h->stream), "sparse: scratch");
    cudaError_t e = launch_sparse_count(h->n, h->flags, counts, h->stream);
    h->launches += 2;
    int nf = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nf, counts + nb, sizeof(int), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { cudaFreeAsync(counts, h->stream); return cuda_fail(h, e, "sparse: count"); }
    for (int b = 0; b < 2; ++b)
        if (h->buf[b]) { cudaFree(h->buf[b]); h->buf[b] = nullptr; }
    if (h->pos) { cudaFree(h->pos); h->pos = nullptr; }
    if (h->nbr) { cudaFree(h->nbr); h->nbr = nullptr; }
    h->nf = nf;
    const size_t nrec = (size_t)(nf > 0 ? nf : 1);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&h->buf[b], nrec * h->node_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->pos, nrec * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->nbr, nrec * (size_t)(h->cfg.q - 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&idx, (size_t)h->n * sizeof(int), h->stream);
    if (e == cudaSuccess) {
        int per[3] = {h->cfg.periodic[0] ? 1 : 0, h->cfg.periodic[1] ? 1 : 0, h->cfg.periodic[2] ? 1 : 0};
        e = launch_sparse_build(h->cfg.q, h->cfg.nx, h->cfg.ny, h->cfg.nz, per, h->flags, counts, idx, h->pos, nf,
                                h->nbr, h->stream);
        h->launches += 2;
    }
    if (idx) cudaFreeAsync(idx, h->stream);
    cudaFreeAsync(counts, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sparse: fluid list");
    return LBM_OK;
}

// Compact layout: classes the tile columns of the row-pair variant
// h->variant by their fluid counts (counted once per geometry and variant)
// with threshold h->cthr and uploads the two lists; the node list is written
// by a kernel from the flags.
lbm_status build_compact(lbm_tau1* h)
{
    const lbm_tau1_config& c = h->cfg;
    h->ctile = compact_tiles(c.q, c.storage, h->variant);
    const CompactTiles& ct = h->ctile;
    const int64_t nb = compact_tile_columns(ct, c.nx, c.ny, c.nz);
    if (h->ccounted != h->variant) {
        if (nb > h->ccap) {
            for (int** p : {&h->ccounts, &h->ctiles, &h->clisted})
                if (*p) { cudaFree(*p); *p = nullptr; }
            h->ccap = 0;
            LBM_CUDA(h, cudaMalloc((void**)&h->ccounts, (size_t)nb * sizeof(int)), "compact: counts");
            LBM_CUDA(h, cudaMalloc((void**)&h->ctiles, (size_t)nb * sizeof(int)), "compact: tile list");
            LBM_CUDA(h, cudaMalloc((void**)&h->clisted, (size_t)2 * nb * sizeof(int)), "compact: listed columns");
            h->ccap = nb;
        }
        LBM_CUDA(h, launch_compact_count(ct, c.nx, c.ny, c.nz, h->flags, h->ccounts, h->stream),
                 "compact: count kernel");
        ++h->launches;
        h->ccounts_host.assign((size_t)nb, 0);
        LBM_CUDA(h, cudaMemcpyAsync(h->ccounts_host.data(), h->ccounts, (size_t)nb * sizeof(int),
                                    cudaMemcpyDefault, h->stream), "compact: counts copy");
        LBM_CUDA(h, cudaStreamSynchronize(h->stream), "compact: counts sync");
        if (!h->cnodes) {  // the fluid nodes of the geometry: the longest node list
            int64_t nf = 0;
            for (int v : h->ccounts_host) nf += v;
            LBM_CUDA(h, cudaMalloc((void**)&h->cnodes, (size_t)(nf > 0 ? nf : 1) * sizeof(int)),
                     "compact: node list");
        }
        StepArgs a;
        fill_args(h, a);
        h->c_tiled_ok = tau1_rowpair_ok(c.q, c.storage, ct.shape, a);
        if (h->c_tiled_ok && !h->cside) {
            LBM_CUDA(h, cudaStreamCreateWithFlags(&h->cside, cudaStreamNonBlocking), "compact: side stream");
            LBM_CUDA(h, cudaEventCreateWithFlags(&h->cfork, cudaEventDisableTiming), "compact: event");
            LBM_CUDA(h, cudaEventCreateWithFlags(&h->cjoin, cudaEventDisableTiming), "compact: event");
        }
        h->ccounted = h->variant;
    }
    std::vector<int> tiles, listed, offsets;
    int64_t nodes = 0;
    h->c_tiled_fluid = 0;
    h->c_empty = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int cnt = h->ccounts_host[(size_t)b];
        if (cnt == 0) { ++h->c_empty; continue; }
        const double m = (double)compact_tile_nodes(ct, c.nx, c.ny, c.nz, (int)b);
        if (h->c_tiled_ok && (double)cnt >= h->cthr * m) {
            tiles.push_back((int)b);
            h->c_tiled_fluid += cnt;
        } else {
            listed.push_back((int)b);
            offsets.push_back((int)nodes);
            nodes += cnt;
        }
    }
    listed.insert(listed.end(), offsets.begin(), offsets.end());
    h->n_ctiles = (int64_t)tiles.size();
    h->n_clisted = (int64_t)offsets.size();
    h->n_cnodes = nodes;
    if (!tiles.empty())
        LBM_CUDA(h, cudaMemcpyAsync(h->ctiles, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyDefault,
                                    h->stream), "compact: tile list copy");
    if (!listed.empty())
        LBM_CUDA(h, cudaMemcpyAsync(h->clisted, listed.data(), listed.size() * sizeof(int), cudaMemcpyDefault,
                                    h->stream), "compact: listed columns copy");
    LBM_CUDA(h, launch_compact_nodes(ct, c.nx, c.ny, c.nz, h->flags, h->clisted, h->clisted + h->n_clisted,
                                     (int)h->n_clisted, h->cnodes, h->stream),
             "compact: node list kernel");
    if (h->n_clisted) ++h->launches;
    // the host vectors are copied from before they go out of scope
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "compact: lists sync");
    return LBM_OK;
}

// Kernel launches of one step of the main kernel(s).
int step_launches(const lbm_tau1* h)
{
    if (!h->compact) return 1;
    return (h->n_ctiles > 0 ? 1 : 0) + (h->n_cnodes > 0 ? 1 : 0);
}

cudaError_t launch_kernel(const lbm_tau1* h, int variant, const StepArgs& a)
{
    if (h->cfg.q == LBM_D2Q9) return launch_tau1_2d(h->kernel == LBM_KERNEL_SIMPLE, h->cfg.storage, a, h->stream);
    if (h->compact) {
        // Disjoint node sets, both read from the same copy: with both lists
        // non-empty the node-list kernel runs on a side stream forked from
        // and joined back into the handle's stream, so that the two kernels
        // overlap (each fills the SMs the other's tail leaves idle).
        const bool both = h->n_ctiles > 0 && h->n_cnodes > 0;
        cudaStream_t ls = both ? h->cside : h->stream;
        cudaError_t e = cudaSuccess;
        if (both) {
            e = cudaEventRecord(h->cfork, h->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cside, h->cfork, 0);
        }
        if (e == cudaSuccess) e = launch_tau1_list(h->cfg.q, h->cfg.storage, a, h->cnodes, h->n_cnodes, ls);
        if (e == cudaSuccess && both) e = cudaEventRecord(h->cjoin, h->cside);
        if (e == cudaSuccess)
            e = launch_tau1_rowpair_list(h->cfg.q, h->cfg.storage, h->ctile.shape, h->ctile.zchunk, a, h->ctiles,
                                         (int)h->n_ctiles, h->stream);
        if (e == cudaSuccess && both) e = cudaStreamWaitEvent(h->stream, h->cjoin, 0);
        return e;
    }
    if (h->sparse) return launch_tau1_sparse(h->cfg.q, h->cfg.storage, a, (int)h->nf, h->nbr, h->stream);
    if (h->kernel == LBM_KERNEL_TILED) return launch_tau1_tiled(h->cfg.q, h->cfg.storage, variant, a, h->stream);
    return launch_tau1_simple(h->cfg.q, h->cfg.storage, a, h->stream);
}

lbm_status launch_step(lbm_tau1* h)
{
    StepArgs a;
    fill_args(h, a);
    if (h->bgk) {
        cudaError_t e = launch_bgk_step(h->cfg.q, h->cfg.storage, a, h->fbuf[h->fcur], h->fbuf[h->fcur ^ 1],
                                        h->bgk_mask, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "bgk step launch");
        ++h->launches;
        h->fcur ^= 1;
        ++h->step;
        return LBM_OK;
    }
    cudaError_t e = launch_kernel(h, h->variant, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "tau1 step launch");
    h->launches += step_launches(h);
    if (h->p_axis >= 0) {
        e = launch_zou_he(h->cfg.q, h->cfg.storage, a, h->p_axis, h->p_lo, h->p_hi, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "pressure-face launch");
        ++h->launches;
    }
    h->cur ^= 1;
    ++h->step;
    if (h->dscale && h->step % RESCALE_EVERY == 0) {
        const int64_t nb = (rescale_scratch_floats(h->n) - 4) / 4;
        e = launch_rescale(h->cfg.storage, h->sparse ? h->nf : h->n, h->buf[h->cur], h->sparse ? nullptr : h->flags,
                           h->dscale, h->rescale_scratch, h->rescale_scratch + 4 * nb, gmax_of(h), h->stream);
        h->launches += 3;
        if (e != cudaSuccess) return cuda_fail(h, e, "rescale kernels");
    }
    return LBM_OK;
}

// Compact layout: mean time of `trials` step launches (after one warm-up)
// of the current lists; the launches rewrite only the scratch copy.
lbm_status time_compact(lbm_tau1* h, int trials, cudaEvent_t e0, cudaEvent_t e1, float* ms)
{
    StepArgs a;
    fill_args(h, a);
    cudaError_t e = launch_kernel(h, 0, a);
    h->launches += step_launches(h);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int t = 0; t < trials && e == cudaSuccess; ++t) {
        e = launch_kernel(h, 0, a);
        h->launches += step_launches(h);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune: trial");
    *ms /= (float)trials;
    return LBM_OK;
}

// Compact layout: times every pair of a row-pair variant and a threshold of
// LBM_TAU1_COMPACT_THRESHOLDS and keeps the fastest pair.
lbm_status autotune_compact(lbm_tau1* h, int trials, int32_t* chosen, float* ms_per_step)
{
    static const double thr[] = LBM_TAU1_COMPACT_THRESHOLDS;
    const int nt = (int)(sizeof(thr) / sizeof(thr[0]));
    cudaEvent_t e0, e1;
    LBM_CUDA(h, cudaEventCreate(&e0), "autotune: event");
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(h, e, "autotune: event"); }
    lbm_status st = LBM_OK;
    int best_v = h->variant, best_t = 0;
    float best_ms = -1.f;
    for (int v = 0; v < variant_count(h) && st == LBM_OK; ++v) {
        for (int t = 0; t < nt && st == LBM_OK; ++t) {
            h->variant = v;
            h->cthr = thr[t];
            float ms = 0.f;
            st = build_compact(h);
            if (st == LBM_OK) st = time_compact(h, trials, e0, e1, &ms);
            if (st == LBM_OK && (best_ms < 0.f || ms < best_ms)) {
                best_v = v;
                best_t = t;
                best_ms = ms;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    h->variant = best_v;
    h->cthr = thr[best_t];
    if (lbm_status s2 = build_compact(h)) return s2;
    if (chosen) *chosen = best_t;
    if (ms_per_step) *ms_per_step = best_ms;
    return LBM_OK;
}

}  // namespace

void lbm::set_create_error(const std::string& msg) { g_create_error = msg; }

lbm_status lbm::fill_stats(const double* r, int64_t n_nodes, const double g[3], int64_t step, lbm_tau1_stats* out)
{
    std::memset(out, 0, sizeof(*out));
    out->step = step;
    out->n_nodes = n_nodes;
    out->n_fluid = (int64_t)r[RED_NFLUID];
    out->nonfinite = (int64_t)r[RED_NONFINITE];
    out->drho_sum = r[RED_DRHO];
    out->mass = (double)out->n_fluid + r[RED_DRHO];
    out->mean_ux_superficial = r[RED_PX] / (double)n_nodes;
    const double nf = out->n_fluid > 0 ? (double)out->n_fluid : 1.0;
    out->mean_u_fluid[0] = r[RED_PX] / nf;
    out->mean_u_fluid[1] = r[RED_PY] / nf;
    out->mean_u_fluid[2] = r[RED_PZ] / nf;
    out->max_abs_u = r[RED_UMAX];
    out->permeability = g[0] != 0.0 ? (1.0 / 6.0) * out->mean_ux_superficial / g[0] : NAN;
    return (out->nonfinite > 0 || out->max_abs_u > 0.3) ? LBM_EDIVERGED : LBM_OK;
}

extern "C" {

int32_t lbm_tau1_abi_version(void) { return LBM_TAU1_ABI_VERSION; }

const char* lbm_tau1_last_error(const lbm_tau1* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int64_t lbm_tau1_launch_count(const lbm_tau1* h) { return h ? h->launches : 0; }

lbm_status lbm_tau1_create(const lbm_tau1_config* cfg, lbm_tau1** out)
{
    if (out) *out = nullptr;
    if (!cfg || !out) return fail(nullptr, LBM_EINVAL, "create: NULL argument");
    if (cfg->q != LBM_D2Q9 && cfg->q != 19 && cfg->q != 27)
        return fail(nullptr, LBM_EINVAL, "create: q must be 9, 19 or 27");
    if (cfg->q == LBM_D2Q9 && (cfg->nz != 1 || cfg->layout != LBM_DENSE || cfg->scheme != LBM_SCHEME_TAU1))
        return fail(nullptr, LBM_EINVAL, "create: D2Q9 takes one plane (nz = 1), the dense layout and the Tau1 scheme");
    if (storage_node_bytes(cfg->storage) == 0) return fail(nullptr, LBM_EINVAL, "create: bad storage");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return fail(nullptr, LBM_EINVAL, "create: box sizes must be >= 1");
    if (cfg->layout != LBM_DENSE && cfg->layout != LBM_SPARSE && cfg->layout != LBM_COMPACT)
        return fail(nullptr, LBM_EINVAL, "create: bad layout");
    if (cfg->layout != LBM_DENSE && cfg->scheme != LBM_SCHEME_TAU1)
        return fail(nullptr, LBM_EINVAL, "create: the sparse and compact layouts are for the Tau1 scheme");
    if (cfg->layout != LBM_DENSE && (int64_t)cfg->nx * cfg->ny * cfg->nz >= ((int64_t)1 << 31))
        return fail(nullptr, LBM_EINVAL, "create: the sparse and compact layouts take boxes of fewer than 2^31 nodes");
    if (cfg->scheme != LBM_SCHEME_TAU1 && cfg->scheme != LBM_SCHEME_BGK)
        return fail(nullptr, LBM_EINVAL, "create: bad scheme");
    if (cfg->scheme == LBM_SCHEME_BGK && !bgk_supported(cfg->q, cfg->storage))
        return fail(nullptr, LBM_EINVAL, "create: the BGK scheme supports LBM_F32 and LBM_F64 storage");
    if (cfg->kernel > LBM_KERNEL_TILED) return fail(nullptr, LBM_EINVAL, "create: bad kernel");
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(cfg->g[d])) return fail(nullptr, LBM_EINVAL, "create: g must be finite");
    const int64_t n = (int64_t)cfg->nx * cfg->ny * cfg->nz;
    if (n > ((int64_t)1 << 33)) return fail(nullptr, LBM_EINVAL, "create: box too large");

    lbm_tau1* h = new (std::nothrow) lbm_tau1();
    if (!h) return fail(nullptr, LBM_ENOMEM, "create: host allocation failed");
    h->cfg = *cfg;
    h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    h->n = n;
    h->node_bytes = storage_node_bytes(cfg->storage);
    h->kernel = cfg->kernel;
    h->sparse = cfg->layout == LBM_SPARSE;
    h->compact = cfg->layout == LBM_COMPACT;
    // one thread per fluid node, or the compact split: no tile variants
    if (h->sparse || h->compact) h->kernel = LBM_KERNEL_SIMPLE;
    const bool tiled_ok = cfg->q == LBM_D2Q9 || tau1_tiled_supported(cfg->q, cfg->storage, n);
    if (h->kernel == LBM_KERNEL_AUTO) h->kernel = tiled_ok ? LBM_KERNEL_TILED : LBM_KERNEL_SIMPLE;
    if (h->kernel == LBM_KERNEL_TILED && !tiled_ok) {
        delete h;
        return fail(nullptr, LBM_EINVAL, "create: tiled kernel not available for this lattice/storage");
    }
    cudaError_t e = cudaSuccess;
    h->bgk = cfg->scheme == LBM_SCHEME_BGK;
    // dense: two copies of the box; sparse: allocated by set_geometry (nf records)
    // (compact: one more record, the solid sentinel of the node-list kernel)
    for (int b = 0; b < 2 && e == cudaSuccess && !h->sparse; ++b)
        e = cudaMalloc(&h->buf[b], (size_t)(n + (h->compact ? 1 : 0)) * h->node_bytes);
    if (h->bgk)
        for (int b = 0; b < 2 && e == cudaSuccess; ++b)
            e = cudaMalloc(&h->fbuf[b], (size_t)n * cfg->q * (cfg->storage == LBM_F64 ? 8 : 4));
    if (h->bgk && e == cudaSuccess) e = cudaMalloc((void**)&h->bgk_mask, (size_t)n * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->flags, (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&h->red_partials, (size_t)reduce_blocks(n) * RED_FIELDS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->red_out, RED_FIELDS * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h->red_host, RED_FIELDS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dtimeouts, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dtimeouts, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess && sixteen(h)) e = cudaMalloc(&h->dscale, 8 * sizeof(float));
    if (e == cudaSuccess && sixteen(h))
        e = cudaMalloc(&h->rescale_scratch, (size_t)rescale_scratch_floats(n) * sizeof(float));
    if (e != cudaSuccess) {
        lbm_status st = cuda_fail(nullptr, e, "create: device allocation");
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_tau1_destroy(lbm_tau1* h)
{
    if (!h) return LBM_OK;
    free_all(h);
    delete h;
    return LBM_OK;
}

lbm_status lbm_tau1_synchronize(lbm_tau1* h)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "synchronize: NULL handle");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
    if (unsigned t = take_timeouts(h))
        return fail(h, LBM_ETIMEOUT, "synchronize: " + std::to_string(t) + " staged-copy waits ran out");
    return LBM_OK;
}

lbm_status lbm_tau1_set_geometry(lbm_tau1* h, const uint8_t* solid, int on_device)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "set_geometry: NULL handle");
    if (!solid) return fail(h, LBM_EINVAL, "set_geometry: NULL mask");
    if (lbm_status st = check_ptr(h, solid, on_device, "set_geometry mask")) return st;
    const uint8_t* dsolid = solid;
    uint8_t* tmp = nullptr;
    if (!on_device) {
        LBM_CUDA(h, cudaMallocAsync((void**)&tmp, (size_t)h->n, h->stream), "set_geometry: staging allocation");
        LBM_CUDA(h, cudaMemcpyAsync(tmp, solid, (size_t)h->n, cudaMemcpyDefault, h->stream), "set_geometry: copy");
        dsolid = tmp;
    }
    int per[3] = {h->cfg.periodic[0] ? 1 : 0, h->cfg.periodic[1] ? 1 : 0, h->cfg.periodic[2] ? 1 : 0};
    cudaError_t e = launch_build_flags(h->cfg.q, h->cfg.nx, h->cfg.ny, h->cfg.nz, per, dsolid, h->flags, h->stream);
    ++h->launches;
    if (tmp) cudaFreeAsync(tmp, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_geometry: flags kernel");
    if (h->sparse)
        if (lbm_status st = build_fluid_list(h)) return st;
    if (h->compact) {
        // a new geometry: count again, and size the node list again
        h->ccounted = -1;
        if (h->cnodes) { cudaFree(h->cnodes); h->cnodes = nullptr; }
        if (lbm_status st = build_compact(h)) return st;
    }
    const double zero[4] = {0, 0, 0, 0};
    set_scales(h, zero);
    if (lbm_status st = upload_scales(h)) return st;
    for (int b = 0; b < 2; ++b) {
        // drho = 0, u = 0 on fluid nodes; solid nodes marked with drho = NaN
        if (h->sparse) e = launch_import_sparse(h->cfg.storage, (int)h->nf, nullptr, h->pos, h->buf[b], h->scale, h->stream);
        else e = launch_import_state(h->cfg.storage, h->n, nullptr, h->buf[b], h->flags, h->scale, h->stream);
        ++h->launches;
        if (e == cudaSuccess && h->compact) {
            e = launch_compact_sentinel(h->cfg.storage, h->buf[b], h->n, h->dscale, h->stream);
            ++h->launches;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "set_geometry: state init");
    }
    h->cur = 0;
    h->fcur = 0;
    h->step = 0;
    h->n_fluid = -1;
    h->has_geometry = true;
    return bgk_from_state(h);
}

lbm_status lbm_tau1_set_fields(lbm_tau1* h, const double* drho, const double* ux, const double* uy,
                               const double* uz, int on_device)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "set_fields: NULL handle");
    if (!h->has_geometry) return fail(h, LBM_ESTATE, "set_fields: call set_geometry first");
    const double* src[4] = {drho, ux, uy, uz};
    for (int f = 0; f < 4; ++f) {
        if (!src[f]) return fail(h, LBM_EINVAL, "set_fields: NULL field");
        if (lbm_status st = check_ptr(h, src[f], on_device, "set_fields field")) return st;
    }
    const size_t bytes = (size_t)h->n * sizeof(double);
    double* tmp = nullptr;
    const double* dsrc[4];
    if (!on_device) {
        LBM_CUDA(h, cudaMallocAsync((void**)&tmp, 4 * bytes, h->stream), "set_fields: staging allocation");
        for (int f = 0; f < 4; ++f) {
            LBM_CUDA(h, cudaMemcpyAsync(tmp + f * h->n, src[f], bytes, cudaMemcpyDefault, h->stream),
                     "set_fields: copy");
            dsrc[f] = tmp + f * h->n;
        }
    } else {
        for (int f = 0; f < 4; ++f) dsrc[f] = src[f];
    }
    if (h->cfg.storage == LBM_F16S || h->cfg.storage == LBM_BF16S) {
        // power-of-two scale putting the largest |value| near 2^12 (FP16 max ~2^16)
        int blocks = reduce_blocks(h->n);
        cudaError_t e = launch_absmax_f64(h->n, dsrc, h->flags, h->red_out, h->red_partials, blocks, h->stream);
        h->launches += 2;
        if (e != cudaSuccess) return cuda_fail(h, e, "set_fields: absmax");
        LBM_CUDA(h, cudaMemcpyAsync(h->red_host, h->red_out, 4 * sizeof(double), cudaMemcpyDefault, h->stream),
                 "set_fields: absmax copy");
        LBM_CUDA(h, cudaStreamSynchronize(h->stream), "set_fields: sync");
        set_scales(h, h->red_host);
        if (lbm_status st = upload_scales(h)) return st;
    }
    cudaError_t e = h->sparse
                        ? launch_import_sparse(h->cfg.storage, (int)h->nf, dsrc, h->pos, h->buf[h->cur], h->scale,
                                               h->stream)
                        : launch_import_state(h->cfg.storage, h->n, dsrc, h->buf[h->cur], h->flags, h->scale, h->stream);
    ++h->launches;
    if (tmp) cudaFreeAsync(tmp, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_fields: import kernel");
    h->step = 0;
    return bgk_from_state(h);
}

lbm_status lbm_tau1_get_fields(lbm_tau1* h, double* drho, double* ux, double* uy, double* uz, int on_device)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "get_fields: NULL handle");
    if (!h->has_geometry) return fail(h, LBM_ESTATE, "get_fields: call set_geometry first");
    double* dst[4] = {drho, ux, uy, uz};
    for (int f = 0; f < 4; ++f)
        if (lbm_status st = check_ptr(h, dst[f], on_device, "get_fields field")) return st;
    if (lbm_status st = bgk_refresh_state(h)) return st;
    if (lbm_status st = download_scales(h)) return st;
    const size_t bytes = (size_t)h->n * sizeof(double);
    if (!on_device && !h->sparse) {
        // page-locked host arrays that the GPU can address: the export kernel
        // writes them directly, with no device staging copy
        double* view[4];
        bool direct = true;
        for (int f = 0; f < 4 && direct; ++f) {
            cudaPointerAttributes at;
            view[f] = nullptr;
            if (!dst[f] || cudaPointerGetAttributes(&at, dst[f]) != cudaSuccess) {
                cudaGetLastError();
                direct = false;
            } else if (at.type == cudaMemoryTypeHost && at.devicePointer) {
                view[f] = static_cast<double*>(at.devicePointer);
            } else {
                direct = false;
            }
        }
        if (direct) {
            cudaError_t e = launch_export_state(h->cfg.storage, h->n, h->buf[h->cur], view, h->flags, h->inv_scale,
                                                h->stream);
            ++h->launches;
            if (e != cudaSuccess) return cuda_fail(h, e, "get_fields: export kernel");
            LBM_CUDA(h, cudaStreamSynchronize(h->stream), "get_fields: sync");
            return LBM_OK;
        }
    }
    double* tmp = nullptr;
    LBM_CUDA(h, cudaMallocAsync((void**)&tmp, 4 * bytes, h->stream), "get_fields: staging allocation");
    double* ddst[4];
    for (int f = 0; f < 4; ++f) ddst[f] = (on_device && dst[f]) ? dst[f] : tmp + f * h->n;
    cudaError_t e = cudaSuccess;
    if (h->sparse) {
        // solid nodes report 0: clear, then scatter the list
        for (int f = 0; f < 4 && e == cudaSuccess; ++f)
            if (dst[f] || !on_device) e = cudaMemsetAsync(ddst[f], 0, bytes, h->stream);
        if (e == cudaSuccess)
            e = launch_export_sparse(h->cfg.storage, (int)h->nf, h->buf[h->cur], h->pos, ddst, h->inv_scale, h->stream);
    } else {
        e = launch_export_state(h->cfg.storage, h->n, h->buf[h->cur], ddst, h->flags, h->inv_scale, h->stream);
    }
    ++h->launches;
    if (e != cudaSuccess) { cudaFreeAsync(tmp, h->stream); return cuda_fail(h, e, "get_fields: export kernel"); }
    if (!on_device) {
        for (int f = 0; f < 4; ++f)
            if (dst[f]) {
                e = cudaMemcpyAsync(dst[f], ddst[f], bytes, cudaMemcpyDefault, h->stream);
                if (e != cudaSuccess) { cudaFreeAsync(tmp, h->stream); return cuda_fail(h, e, "get_fields: copy"); }
            }
    }
    cudaFreeAsync(tmp, h->stream);
    if (!on_device) LBM_CUDA(h, cudaStreamSynchronize(h->stream), "get_fields: sync");
    return LBM_OK;
}

lbm_status lbm_tau1_step(lbm_tau1* h, int64_t nsteps)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "step: NULL handle");
    if (nsteps < 0) return fail(h, LBM_EINVAL, "step: nsteps < 0");
    if (!h->has_geometry) return fail(h, LBM_ESTATE, "step: call set_geometry first");
    for (int64_t t = 0; t < nsteps; ++t)
        if (lbm_status st = launch_step(h)) return st;
    return LBM_OK;
}

lbm_status lbm_tau1_set_pressure(lbm_tau1* h, int32_t axis, double rho_lo, double rho_hi)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "set_pressure: NULL handle");
    if (axis < 0) {
        h->p_axis = -1;
        return LBM_OK;
    }
    const int dims = h->cfg.q == LBM_D2Q9 ? 2 : 3;
    if (axis >= dims) return fail(h, LBM_EINVAL, "set_pressure: axis out of range");
    if (h->cfg.periodic[axis]) return fail(h, LBM_EINVAL, "set_pressure: the axis must not be periodic");
    if (h->sparse || h->bgk) return fail(h, LBM_EINVAL, "set_pressure: dense layout and Tau1 scheme only");
    if (!(std::isfinite(rho_lo) && std::isfinite(rho_hi) && rho_lo > 0.0 && rho_hi > 0.0))
        return fail(h, LBM_EINVAL, "set_pressure: densities must be finite and positive");
    h->p_axis = axis;
    h->p_lo = rho_lo;
    h->p_hi = rho_hi;
    return LBM_OK;
}

lbm_status lbm_tau1_copy_plane(lbm_tau1* h, int32_t z, void* buf, int32_t to_handle)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "copy_plane: NULL handle");
    if (!buf) return fail(h, LBM_EINVAL, "copy_plane: NULL buffer");
    if (h->sparse || h->bgk) return fail(h, LBM_EINVAL, "copy_plane: dense layout and Tau1 scheme only");
    if (h->cfg.storage == LBM_F16S)
        return fail(h, LBM_EINVAL, "copy_plane: FP16 records carry the handle's own scales; use F32, F64 or BF16S");
    if (z < 0 || z >= h->cfg.nz) return fail(h, LBM_EINVAL, "copy_plane: plane out of range");
    if (!h->has_geometry) return fail(h, LBM_ESTATE, "copy_plane: call set_geometry first");
    if (lbm_status st = check_ptr(h, buf, 1, "copy_plane buffer")) return st;
    const size_t plane = (size_t)h->cfg.nx * (size_t)h->cfg.ny * h->node_bytes;
    unsigned char* base = static_cast<unsigned char*>(h->buf[h->cur]) + (size_t)z * plane;
    LBM_CUDA(h, cudaMemcpyAsync(to_handle ? static_cast<void*>(base) : buf, to_handle ? buf : base, plane,
                                cudaMemcpyDeviceToDevice, h->stream), "copy_plane: copy");
    return LBM_OK;
}

int32_t lbm_tau1_variant_count(const lbm_tau1* h) { return h ? variant_count(h) : 0; }

lbm_status lbm_tau1_set_variant(lbm_tau1* h, int32_t variant)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "set_variant: NULL handle");
    if (variant < 0 || variant >= variant_count(h)) return fail(h, LBM_EINVAL, "set_variant: no such variant");
    h->variant = variant;
    return (h->compact && h->has_geometry) ? build_compact(h) : LBM_OK;
}

lbm_status lbm_tau1_selftest_timeout(lbm_tau1* h)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "selftest_timeout: NULL handle");
    LBM_CUDA(h, launch_selftest_timeout(h->dtimeouts, h->stream), "selftest_timeout: launch");
    ++h->launches;
    return LBM_OK;
}

lbm_status lbm_tau1_set_compact_threshold(lbm_tau1* h, double f)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "set_compact_threshold: NULL handle");
    if (!h->compact) return fail(h, LBM_EINVAL, "set_compact_threshold: not the compact layout");
    if (!(f >= 0.0 && f <= 1.01)) return fail(h, LBM_EINVAL, "set_compact_threshold: f outside [0, 1.01]");
    h->cthr = f;
    return h->has_geometry ? build_compact(h) : LBM_OK;
}

lbm_status lbm_tau1_get_compact_info(const lbm_tau1* h, lbm_tau1_compact_info* out)
{
    if (!h || !out) return fail(const_cast<lbm_tau1*>(h), LBM_EINVAL, "get_compact_info: NULL argument");
    lbm_tau1* hm = const_cast<lbm_tau1*>(h);
    if (!h->compact) return fail(hm, LBM_EINVAL, "get_compact_info: not the compact layout");
    if (!h->has_geometry) return fail(hm, LBM_ESTATE, "get_compact_info: call set_geometry first");
    const lbm_tau1_config& c = h->cfg;
    std::memset(out, 0, sizeof(*out));
    out->threshold = h->cthr;
    out->variant = h->variant;
    out->tile[0] = 32;
    out->tile[1] = h->ctile.h;
    out->tile[2] = c.nz < h->ctile.zchunk ? c.nz : h->ctile.zchunk;
    out->tiled_ok = h->c_tiled_ok ? 1 : 0;
    out->columns = (int64_t)h->ccounts_host.size();
    out->empty_columns = h->c_empty;
    out->tiled_columns = h->n_ctiles;
    out->listed_columns = h->n_clisted;
    int64_t tn = 0;
    for (size_t b = 0; b < h->ccounts_host.size(); ++b) {
        const int cnt = h->ccounts_host[b];
        const int64_t m = compact_tile_nodes(h->ctile, c.nx, c.ny, c.nz, (int)b);
        if (cnt == m) ++out->full_columns;
        if (h->c_tiled_ok && cnt > 0 && (double)cnt >= h->cthr * (double)m) tn += m;
    }
    out->tiled_nodes = tn;
    out->tiled_fluid = h->c_tiled_fluid;
    out->listed_nodes = h->n_cnodes;
    return LBM_OK;
}

lbm_status lbm_tau1_autotune(lbm_tau1* h, int32_t trials, int32_t* chosen, float* ms_per_step)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "autotune: NULL handle");
    if (trials < 1) return fail(h, LBM_EINVAL, "autotune: trials < 1");
    if (!h->has_geometry) return fail(h, LBM_ESTATE, "autotune: call set_geometry first");
    if (h->bgk) {
        if (chosen) *chosen = 0;
        if (ms_per_step) *ms_per_step = 0.f;
        return LBM_OK;
    }
    if (h->compact) return autotune_compact(h, trials, chosen, ms_per_step);
    const std::string key = tune_key(h);
    int cached = 0;
    double cached_ms = 0;
    if (tune_cache_lookup(key, &cached, &cached_ms) && cached >= 0 && cached < variant_count(h)) {
        h->variant = cached;
        if (chosen) *chosen = cached;
        if (ms_per_step) *ms_per_step = (float)cached_ms;
        return LBM_OK;
    }
    // Every trial launch reads the current copy and rewrites the other one
    // without swapping, so the state is left as it was.
    StepArgs a;
    fill_args(h, a);
    cudaEvent_t e0, e1;
    LBM_CUDA(h, cudaEventCreate(&e0), "autotune: event");
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(h, e, "autotune: event"); }
    const int nv = variant_count(h);
    int best = h->variant;
    float best_ms = 0.f;
    for (int v = 0; v < nv && e == cudaSuccess; ++v) {
        e = launch_kernel(h, v, a);  // warm-up (and first-use set-up)
        ++h->launches;
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int t = 0; t < trials && e == cudaSuccess; ++t) {
            e = launch_kernel(h, v, a);
            ++h->launches;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)trials;
        if (e == cudaSuccess && (v == 0 || ms < best_ms)) { best = v; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune: trial");
    h->variant = best;
    if (chosen) *chosen = best;
    if (ms_per_step) *ms_per_step = best_ms;
    tune_cache_store(key, best, best_ms);
    return LBM_OK;
}

void lbm_tau1_set_tune_cache(const char* path) { tune_cache_set_path(path); }

lbm_status lbm_tau1_reduce(lbm_tau1* h, lbm_tau1_stats* out)
{
    if (!h) return fail(nullptr, LBM_EINVAL, "reduce: NULL handle");
    if (!out) return fail(h, LBM_EINVAL, "reduce: NULL output");
    if (!h->has_geometry) return fail(h, LBM_ESTATE, "reduce: call set_geometry first");
    if (lbm_status st = bgk_refresh_state(h)) return st;
    if (lbm_status st = download_scales(h)) return st;
    const void* f[4] = {h->buf[h->cur], nullptr, nullptr, nullptr};
    cudaError_t e = launch_reduce(h->cfg.storage, true, h->sparse ? h->nf : h->n, f, h->inv_scale,
                                  h->sparse ? nullptr : h->flags, h->cfg.g, h->red_partials,
                                  h->red_out, h->stream);
    h->launches += 2;
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce: kernel");
    LBM_CUDA(h, cudaMemcpyAsync(h->red_host, h->red_out, RED_FIELDS * sizeof(double), cudaMemcpyDefault,
                                h->stream), "reduce: copy");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "reduce: sync");
    if (unsigned t = take_timeouts(h))
        return fail(h, LBM_ETIMEOUT, "reduce: " + std::to_string(t) + " staged-copy waits ran out");
    const lbm_status st = fill_stats(h->red_host, h->n, h->cfg.g, h->step, out);
    h->n_fluid = out->n_fluid;
    if (st == LBM_EDIVERGED) return fail(h, st, "reduce: state diverged (non-finite value or |u| > 0.3)");
    return LBM_OK;
}

}  // extern "C"

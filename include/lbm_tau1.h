/*
 * lbm_tau1.h - C ABI of the GB300 Tau1 lattice Boltzmann solver.
 *
 * Tau1 (Bacza, Tomczak, Matyka, arXiv 2312.14742, Section 2.1, Eq. LBMTau1)
 * is the BGK lattice Boltzmann method at relaxation time tau = 1, where the
 * post-streaming populations equal the equilibria of the neighbours:
 *     f_k(x, t+1) = f_k^eq(rho(x - c_k, t), u(x - c_k, t)).
 * Only rho and u are stored (two ping-pong copies, Section 2.1.3 "Complexity
 * analysis": 2 (d+1) s bytes per node). Each step gathers rho, u of the
 * neighbours x - c_k, forms f_k^eq (Eq. feq, c_s^2 = 1/3), accumulates the
 * new density and momentum, and multiplies the momentum once by 1/rho
 * (Algorithm "Optimized Tau1 algorithm that stores velocity").
 * Walls use halfway bounce-back from the node's own previous (rho*, u*)
 * (Algorithm "Complete Tau1 algorithm with halfway bounce-back").
 * The viscosity is fixed: nu = c_s^2 (tau - 1/2) = 1/6.
 *
 * Conventions for every entry point:
 *  - Node index i = x + nx*(y + ny*z): x fastest.
 *  - State is reported as drho = rho - 1 and u. Storing rho - 1 instead of
 *    rho keeps the density signal in 32- and 16-bit storage.
 *  - Body force g (lattice units) enters by velocity shift: every
 *    equilibrium is evaluated at v = u + g. The stored u is the momentum of
 *    the arriving populations over rho; the physical velocity is u + g/2.
 *    The force is not in the paper (it drives its channel by pressure).
 *  - A link x - c_k that is solid, or that leaves the box across a
 *    non-periodic axis, is a wall.
 *  - Solid nodes hold drho = 0 and u = 0.
 *  - Every call returns an lbm_status; no C++ exception crosses the ABI. On
 *    failure lbm_tau1_last_error() describes the cause.
 *  - Host arrays passed in are read before the call returns and stay owned
 *    by the caller. Device state belongs to the handle.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - Work is queued on the handle's CUDA stream. Calls that return host data
 *    (get_fields to host, reduce) synchronise that stream.
 */
#ifndef LBM_TAU1_H
#define LBM_TAU1_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_TAU1_ABI_VERSION 1

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* bad argument or configuration */
    LBM_ENOMEM = 2,     /* device or host allocation failed */
    LBM_ECUDA = 3,      /* a CUDA call failed (message in last_error) */
    LBM_EDIVERGED = 4,  /* reduction saw a non-finite value or |u| > 0.3 */
    LBM_ETIMEOUT = 5,   /* a bounded device wait (staged copy) ran out; the step results are unreliable */
    LBM_EBUSY = 6,      /* no room (batch admission) */
    LBM_ESTATE = 7      /* call out of order (e.g. step before set_geometry) */
} lbm_status;

/* D2Q9 is one plane (nz = 1): the paper's 2D lattice (Section 3.1), dense
 * layout and Tau1 scheme only. */
typedef enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19, LBM_D3Q27 = 27 } lbm_lattice;

/* Storage of drho and u in device memory. F16S and BF16S hold each field
 * times a power-of-two scale in 16 bits and compute in FP32. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3 } lbm_storage;

/* DENSE: state records for every node of the box. SPARSE: state records for
 * the fluid nodes only, in a list numbered in box order, with an int32 table
 * of the list index of each link's source (-1 for a wall); the list and the
 * table are built by set_geometry (4 (q-1) + 4 bytes per fluid node). The
 * sparse layout is for the Tau1 scheme, boxes of fewer than 2^31 nodes; its
 * FP32 and FP64 results equal the dense kernels' bits. */
/* COMPACT: the dense records, with each step's work split by tile column
 * (32 x H x 24 or 32 nodes: the tile column of the row-pair variant chosen
 * with lbm_tau1_set_variant, 2R variants as for the dense layout's row-pair
 * kernel, variant 0 by default): tile columns without
 * fluid are never read or written; those whose fluid fraction is at least the
 * threshold f* are stepped by the tiled kernel through a list; the fluid
 * nodes of the others are stepped one thread per node through a 4-byte list
 * of box indices. set_geometry builds the lists (f* = 0.3 unless set by
 * lbm_tau1_set_compact_threshold; lbm_tau1_autotune times a few thresholds).
 * Tau1 scheme, D3Q19 or D3Q27, boxes of fewer than 2^31 nodes; FP32 and FP64
 * results equal the dense kernels' bits (solid nodes keep their marker).
 * Every tile column goes to the node list when nx is not a multiple of 32 or
 * ny not of H. */
typedef enum { LBM_DENSE = 0, LBM_SPARSE = 1, LBM_COMPACT = 2 } lbm_layout;

/* LBM_SCHEME_TAU1 is the method. LBM_SCHEME_BGK is the standard pull BGK at
 * tau = 1 with stored populations in SoA form (Algorithm "Standard LBM",
 * AB layout), kept as the comparison kernel; it supports LBM_F32 and
 * LBM_F64 storage and the dense layout. */
typedef enum { LBM_SCHEME_TAU1 = 0, LBM_SCHEME_BGK = 1 } lbm_scheme;

/* Kernel choice for the dense Tau1 layout. AUTO picks TILED when the box
 * has fewer than 2^31 nodes, else SIMPLE. SIMPLE: one thread per node,
 * neighbours from global memory. TILED: shared-memory exchange of each node's
 * outgoing equilibria in a z-marching tile, two nodes per thread (packed
 * f32x2 lanes for FP32 arithmetic). Both give the same bits. */
typedef enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_SIMPLE = 1, LBM_KERNEL_TILED = 2 } lbm_kernel;

typedef struct lbm_tau1_config {
    int32_t q;            /* lbm_lattice */
    int32_t storage;      /* lbm_storage */
    int32_t layout;       /* lbm_layout */
    int32_t scheme;       /* lbm_scheme */
    int32_t nx, ny, nz;   /* box size, each >= 1 */
    uint8_t periodic[3];  /* 1 = periodic along x, y, z */
    uint8_t kernel;       /* lbm_kernel */
    double g[3];          /* body force per unit mass, lattice units */
    void* cuda_stream;    /* cudaStream_t to queue work on; NULL = legacy default stream */
} lbm_tau1_config;

typedef struct lbm_tau1_stats {
    int64_t step;                /* steps taken since set_geometry / set_fields */
    int64_t n_nodes;             /* nx*ny*nz */
    int64_t n_fluid;             /* fluid nodes */
    int64_t nonfinite;           /* fluid nodes holding a non-finite value */
    double mass;                 /* sum over fluid of rho */
    double drho_sum;             /* sum over fluid of drho (mass - n_fluid, exact) */
    double mean_ux_superficial;  /* sum over fluid of (u_x + g_x/2), divided by n_nodes */
    double mean_u_fluid[3];      /* sum over fluid of (u + g/2), divided by n_fluid */
    double max_abs_u;            /* max over fluid of |u + g/2| */
    double permeability;         /* nu * mean_ux_superficial / g_x, nu = 1/6 (Darcy); NaN if g_x == 0 */
} lbm_tau1_stats;

typedef struct lbm_tau1 lbm_tau1;  /* opaque, owned by the library */

/* ABI version of the loaded library (LBM_TAU1_ABI_VERSION it was built with). */
int32_t lbm_tau1_abi_version(void);

/* Validates cfg, allocates the device state of one box (two copies of the
 * state, one record {drho, ux, uy, uz} per node in the storage type; a
 * uint8 node-flag array; reduction scratch) and returns the handle in *out.
 * Errors: LBM_EINVAL (bad cfg or NULL), LBM_ENOMEM, LBM_ECUDA. On error
 * *out is NULL and lbm_tau1_last_error(NULL) gives the message. */
lbm_status lbm_tau1_create(const lbm_tau1_config* cfg, lbm_tau1** out);

/* Sets the geometry: solid has nx*ny*nz bytes, 1 = solid, 0 = fluid, node
 * index x + nx*(y + ny*z). on_device != 0: solid is a device pointer readable
 * on the handle's stream; else a host pointer. Classifies nodes, builds the
 * kernel's wall-link data and resets the state to drho = 0, u = 0 on every
 * node (the paper's rho = 1, u = 0 start) and the step counter to 0.
 * Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_tau1_set_geometry(lbm_tau1* h, const uint8_t* solid, int on_device);

/* Overwrites the state with drho, ux, uy, uz (nx*ny*nz doubles each, host
 * or device per on_device). Values on solid nodes are ignored (kept 0).
 * For 16-bit storage the per-field scales are chosen from these values.
 * Resets the step counter to 0. Requires set_geometry first (LBM_ESTATE). */
lbm_status lbm_tau1_set_fields(lbm_tau1* h, const double* drho, const double* ux,
                               const double* uy, const double* uz, int on_device);

/* Copies the current state out as doubles (nx*ny*nz each, host or device per
 * on_device). Any pointer may be NULL to skip that field. Host copies
 * synchronise the handle's stream. Host arrays in page-locked memory that
 * the GPU can address (all four given, dense layout) are written directly
 * by the export kernel; other host arrays go through a device staging copy.
 * Requires set_geometry (LBM_ESTATE). */
lbm_status lbm_tau1_get_fields(lbm_tau1* h, double* drho, double* ux, double* uy,
                               double* uz, int on_device);

/* Queues nsteps >= 0 Tau1 steps (or BGK steps for LBM_SCHEME_BGK) on the
 * handle's stream and returns without waiting. Each step reads the current
 * copy and writes the other; the copies swap on the host.
 * Errors: LBM_EINVAL (nsteps < 0), LBM_ESTATE (no geometry), LBM_ECUDA. */
lbm_status lbm_tau1_step(lbm_tau1* h, int64_t nsteps);

/* FP64 global reductions of the current state into *out (see
 * lbm_tau1_stats). Deterministic: a fixed two-pass block tree. Synchronises
 * the handle's stream. Returns LBM_EDIVERGED (with *out filled) when a fluid
 * node is non-finite or max|u + g/2| > 0.3. */
lbm_status lbm_tau1_reduce(lbm_tau1* h, lbm_tau1_stats* out);

/* Waits for all work queued on the handle's stream. Returns LBM_ETIMEOUT if
 * a staged (TMA) copy of a step kernel did not complete within its bounded
 * wait (about one second) since the last check; reduce reports the same. */
lbm_status lbm_tau1_synchronize(lbm_tau1* h);

/* Frees the handle and its device memory (after synchronising). NULL is a no-op. */
lbm_status lbm_tau1_destroy(lbm_tau1* h);

/* Last error message of h, or of the calling thread's last failed create
 * when h is NULL. Never NULL; valid until the next call on h. */
const char* lbm_tau1_last_error(const lbm_tau1* h);

/* Number of device kernel launches queued by this handle since creation. */
int64_t lbm_tau1_launch_count(const lbm_tau1* h);

/* Constant-density (pressure) faces on a non-periodic axis (Section 3.3: the
 * 2D validation channel is driven by rho_in at the inlet and rho_out at the
 * outlet, with the boundary conditions of Zou and He). The fluid nodes of the
 * face at coordinate 0 of `axis` keep density rho_lo and those of the face
 * at n - 1 keep rho_hi; after every step each such node takes the velocity
 * along the axis that the Zou-He relation gives from the populations arriving
 * from inside (its known populations: equilibria of fluid sources, halfway
 * bounce-back at walls), u = s (rho_b - 1 - H0 - 2 Hout) / rho_b with s = +1
 * on the low face and -1 on the high face, H0 and Hout the deviations from
 * the weights summed over the known directions parallel to the face and
 * pointing out of the box; the velocity across the axis is zero. Meant for
 * g = 0 (pressure-driven flow). axis = -1 removes the faces. Dense layout,
 * Tau1 scheme; D2Q9 takes axis 0 or 1. Errors: LBM_EINVAL (axis out of range
 * or periodic, a density not finite and positive, sparse layout or BGK). */
lbm_status lbm_tau1_set_pressure(lbm_tau1* h, int32_t axis, double rho_lo, double rho_hi);

/* Halo exchange of a z-slab decomposition (nodes are independent within a
 * step, Section 2.1.2, so a box split into z-slabs needs, per step, only the
 * plane on each side of every cut). Copies plane z of the current state, as
 * the handle stores it (nx*ny records in the storage format: 32, 16 or 8
 * bytes each, solid nodes marked), between the handle and the device buffer
 * buf of nx*ny*record bytes: to_handle = 0 reads the plane into buf, 1
 * writes buf into the plane. Queued on the handle's stream without waiting.
 * A slab holds its planes plus one halo plane below and one above; before
 * each step the halo planes receive the neighbours' edge planes. Dense
 * layout, Tau1 scheme, F64, F32 or BF16S storage (F16 records carry the
 * handle's own scales). Errors: LBM_EINVAL, LBM_ESTATE (no geometry),
 * LBM_ECUDA. */
lbm_status lbm_tau1_copy_plane(lbm_tau1* h, int32_t z, void* buf, int32_t to_handle);

/* ---- Tile-shape autotuning (no counterpart in the paper, whose CPU kernels
 * fix the chunk shape at compile time, Section 3.2). The tiled kernel of the
 * 3D lattices comes in variants: [0, 2R) the row-pair form (R tile shapes:
 * warps per block, resident blocks per SM; [0, R) step 24 z planes per block,
 * [R, 2R) 32), used when nx is a multiple of 32 and ny of the tile height,
 * else the pair-position form of the same chunk height; [2R, 2R + 2T) the
 * pair-position form (T shapes, same chunk rule), TMA-staged when its tiles
 * are full. All variants give the same bits. The default is variant 0. */

/* Number of variants of the handle's step kernel (1 if it has none). */
int32_t lbm_tau1_variant_count(const lbm_tau1* h);

/* Selects a variant, 0 <= variant < lbm_tau1_variant_count(h). LBM_EINVAL otherwise.
 * Compact layout: the lists are rebuilt now if the geometry is set (waits for
 * the stream); the state is unchanged. */
lbm_status lbm_tau1_set_variant(lbm_tau1* h, int32_t variant);

/* Times every variant for `trials` step launches on the handle's current
 * geometry and state (after one warm-up launch each), selects the fastest
 * and returns its index in *chosen and its time per step in *ms_per_step
 * (either may be NULL). The trial launches rewrite only the scratch copy, so
 * the state and step counter are unchanged. Synchronises the stream.
 * Compact layout: times every pair of a row-pair variant and a threshold f*
 * of LBM_TAU1_COMPACT_THRESHOLDS (rebuilding the lists for each), keeps the
 * fastest pair and returns the threshold's index in that list (the variant
 * is in lbm_tau1_get_compact_info); the cache is not used (the best pair
 * depends on the medium).
 * Errors: LBM_EINVAL (trials < 1), LBM_ESTATE (no geometry), LBM_ECUDA. */
#define LBM_TAU1_COMPACT_THRESHOLDS {0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.7, 1.01}
lbm_status lbm_tau1_autotune(lbm_tau1* h, int32_t trials, int32_t* chosen, float* ms_per_step);

/* Autotune cache for the whole process: path of a JSON file of chosen
 * variants keyed by device name, lattice, storage, layout, size bucket
 * (ceil log2 of nx*ny*nz) and whether the box has full tiles. With a cache
 * set, lbm_tau1_autotune first looks its key up and, when found, selects that
 * variant without timing (returning the stored ms per step); otherwise it
 * times the variants and writes its choice to the file. NULL or "" turns the
 * cache off (the default). The file is read and rewritten on each use. */
void lbm_tau1_set_tune_cache(const char* path);

/* Self-test of the failure detection (no counterpart in the paper): queues
 * on the handle's stream one warp that waits, with the staged kernels'
 * bounded wait (about one second), on an mbarrier phase that nothing
 * completes, and counts the timeout in the handle's counter, as a staged
 * copy that never lands would. The next lbm_tau1_synchronize or
 * lbm_tau1_reduce then returns LBM_ETIMEOUT (and clears the count); nothing
 * faults and the context stays usable. For tests and health checks. */
lbm_status lbm_tau1_selftest_timeout(lbm_tau1* h);

/* Compact layout (LBM_COMPACT): how set_geometry split the box. */
typedef struct lbm_tau1_compact_info {
    double threshold;        /* f*: fluid fraction from which a tile column is tiled */
    int32_t variant;         /* row-pair variant of the tiled kernel (lbm_tau1_set_variant) */
    int32_t tile[3];         /* tile column: 32, H, z chunk (24 or 32, or nz if smaller) */
    int32_t tiled_ok;        /* 1 if the tiled kernel can take tile columns */
    int64_t columns;         /* tile columns of the box */
    int64_t empty_columns;   /* without a fluid node: never visited */
    int64_t full_columns;    /* every node fluid */
    int64_t tiled_columns;   /* stepped by the tiled kernel */
    int64_t listed_columns;  /* whose fluid nodes are in the node list */
    int64_t tiled_nodes;     /* box nodes of the tiled columns */
    int64_t tiled_fluid;     /* fluid nodes among them */
    int64_t listed_nodes;    /* length of the node list */
} lbm_tau1_compact_info;

/* Sets f* (0 <= f <= 1.01; 1.01 sends every non-empty tile column to the
 * node list, 0 every one to the tiled kernel) and rebuilds the lists now if
 * the geometry is set (queued on the handle's stream; waits for it). The
 * state is unchanged. LBM_EINVAL: not the compact layout, f out of range. */
lbm_status lbm_tau1_set_compact_threshold(lbm_tau1* h, double f);

/* Fills *out. LBM_EINVAL: NULL argument or not the compact layout;
 * LBM_ESTATE: no geometry yet. */
lbm_status lbm_tau1_get_compact_info(const lbm_tau1* h, lbm_tau1_compact_info* out);

/* ---- Batches: many boxes stepped together (continuous batching) ----------
 * No counterpart in the paper, which steps one domain at a time. A batch
 * holds up to `capacity` live boxes of one lattice and storage format, each
 * with its own size, periodicity, body force, geometry and state. One step of
 * the batch advances every live box by one Tau1 step in a single persistent
 * kernel launch; runs of `graph_steps` steps are replayed from a captured
 * CUDA graph. Boxes are admitted while their device footprint fits in the
 * batch's budget and released when done; admission and release edit device
 * tables only, so captured graphs stay valid. Every box gives the same bits
 * as it would alone in a batch (its arithmetic, step count, stochastic
 * rounding and 16-bit scales depend on its own state only).
 *
 * 16-bit storage in a batch: each of the two state copies of a box has its own
 * scales; a step decodes with the scales of the copy it reads and encodes
 * with those of the copy it writes. For FP16 the kernel picks the next
 * scales every 64 steps of the box from the maxima it saw while storing
 * (headroom rule: the reference magnitude max(m_f, max m / 16, 64 |g|_max)
 * is put at 2^12 when m_f S > 2^13 or the reference times S < 2^9). */
typedef struct lbm_tau1_batch lbm_tau1_batch;  /* opaque, owned by the library */

typedef struct lbm_tau1_batch_config {
    int32_t q;            /* lbm_lattice of every box */
    int32_t storage;      /* lbm_storage of every box */
    int32_t variant;      /* tile shape, 0 <= variant < lbm_tau1_variant_count of a tiled box / 2 */
    int32_t capacity;     /* most boxes live at once, >= 1 */
    int32_t graph_steps;  /* steps per captured graph (>= 1; 0 = 100) */
    int32_t reserved;
    uint64_t hbm_budget;  /* device bytes the boxes may hold; 0 = 90% of the free memory at create */
    void* cuda_stream;    /* cudaStream_t to queue work on; NULL = legacy default stream */
} lbm_tau1_batch_config;

/* Creates an empty batch. Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA (message
 * in lbm_tau1_last_error(NULL)). */
lbm_status lbm_tau1_batch_create(const lbm_tau1_batch_config* cfg, lbm_tau1_batch** out);

/* Device bytes one box of nx*ny*nz nodes holds in a batch of this storage:
 * two state copies (record bytes per node: 32 F64, 16 F32, 8 F16S/BF16S) and
 * one flag byte per node, each allocation rounded up to 256 bytes. */
uint64_t lbm_tau1_batch_footprint(int32_t storage, int32_t nx, int32_t ny, int32_t nz);

/* Admits a box: cfg gives its size, periodicity and g (cfg->q and
 * cfg->storage must match the batch; layout dense, scheme Tau1; kernel and
 * cuda_stream are ignored); solid is its mask as in lbm_tau1_set_geometry
 * (host or device per on_device). The box starts from drho = 0, u = 0 at
 * step 0 and joins the next step of the batch. Returns its slot in *slot.
 * Errors: LBM_EBUSY (capacity reached, or its footprint exceeds the budget
 * left; nothing changes), LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_tau1_batch_admit(lbm_tau1_batch* b, const lbm_tau1_config* cfg, const uint8_t* solid, int on_device,
                                int32_t* slot);

/* Queues nsteps >= 0 steps of every live box and returns without waiting. */
lbm_status lbm_tau1_batch_step(lbm_tau1_batch* b, int64_t nsteps);

/* FP64 reductions (as lbm_tau1_reduce) of n live boxes slots[0..n-1] into
 * out[0..n-1], with one synchronisation of the stream. Returns
 * LBM_EDIVERGED, with every out[] filled, if any of them diverged. */
lbm_status lbm_tau1_batch_stats(lbm_tau1_batch* b, int32_t n, const int32_t* slots, lbm_tau1_stats* out);

/* The same statistics without waiting: queues the reductions of the n live
 * boxes slots[0..n-1] on the batch's stream, with their copy into page-locked
 * memory of the batch and an event after it, and returns. Steps queued after
 * this call do not change the result: each box is reduced as it stands when
 * its reduction runs, which is after the steps queued before this call. The
 * host can queue the next steps, release and admit boxes, and then take the
 * result with lbm_tau1_batch_stats_wait, which waits for the event only and
 * fills out[0..n-1] in the order of slots (a released box is reduced before
 * its memory is freed: both are ordered on the stream). One queued request at
 * a time: LBM_ESTATE if one is already waiting. Errors: LBM_EINVAL (bad
 * arguments, slot not live), LBM_ECUDA. */
lbm_status lbm_tau1_batch_stats_queue(lbm_tau1_batch* b, int32_t n, const int32_t* slots);

/* The self-test of lbm_tau1_selftest_timeout on the batch's stream and
 * counter: the next lbm_tau1_batch_synchronize, lbm_tau1_batch_stats or
 * lbm_tau1_batch_stats_wait (of statistics queued after it) returns
 * LBM_ETIMEOUT. */
lbm_status lbm_tau1_batch_selftest_timeout(lbm_tau1_batch* b);

/* Waits for the statistics queued by lbm_tau1_batch_stats_queue and fills
 * out[0..n-1] (n as queued). Returns LBM_EDIVERGED, with every out[] filled,
 * if any box diverged; LBM_ETIMEOUT if a staged-copy wait ran out in the
 * steps before the reductions; LBM_ESTATE if nothing was queued. */
lbm_status lbm_tau1_batch_stats_wait(lbm_tau1_batch* b, lbm_tau1_stats* out);

/* State of a live box as doubles, as lbm_tau1_get_fields. */
lbm_status lbm_tau1_batch_get_fields(lbm_tau1_batch* b, int32_t slot, double* drho, double* ux, double* uy,
                                     double* uz, int on_device);

/* Releases a live box: its memory returns to the budget once the queued
 * steps that use it have run. LBM_EINVAL if slot is not live. */
lbm_status lbm_tau1_batch_release(lbm_tau1_batch* b, int32_t slot);

/* Waits for all work queued on the batch's stream. */
lbm_status lbm_tau1_batch_synchronize(lbm_tau1_batch* b);

/* Frees the batch and every box (after synchronising). NULL is a no-op. */
lbm_status lbm_tau1_batch_destroy(lbm_tau1_batch* b);

int32_t lbm_tau1_batch_live(const lbm_tau1_batch* b);           /* live boxes */
uint64_t lbm_tau1_batch_bytes_free(const lbm_tau1_batch* b);    /* budget left */
int64_t lbm_tau1_batch_launch_count(const lbm_tau1_batch* b);   /* kernel launches queued (graph nodes counted) */
const char* lbm_tau1_batch_last_error(const lbm_tau1_batch* b); /* never NULL */

/* ---- Reduction without allocation ------------------------------------------
 * The paper has no counterpart to this entry point; it is a service for
 * callers that cannot allocate device memory: code that works from a fixed
 * device arena it manages itself, or inside a framework whose allocator must
 * account for all device memory, and code that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause. It runs the reduction of
 * lbm_tau1_reduce on caller-owned arrays and calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *
 * Scratch: a static device array of LBM_TAU1_NOALLOC_MAX_BLOCKS rows of 8
 * doubles (64 KiB) that every GPU loading this library holds until the
 * process exits. All calls on a device share it; each call overwrites the
 * rows it reads, so nothing carries over between calls. Calls whose work
 * overlaps on the GPU (streams with no ordering between them) race on it.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture. The cached address does not survive cudaDeviceReset of that
 * device: do not call this entry point on a device after resetting it.
 *
 * Arguments: storage (lbm_storage) and n = number of nodes; drho, ux, uy, uz
 * = device arrays of n values in that storage format; inv_scale = host array
 * of 4 floats (16-bit storage: value = stored * inv_scale; NULL = all 1);
 * solid = device array of n bytes, bit 0 set = solid; g = host array of 3
 * doubles (body force, for the physical velocity u + g/2); out = device
 * array of 8 doubles receiving, in order: fluid count, sum drho, sum of the
 * three physical velocity components, max |u + g/2|, non-finite count, 0
 * (the raw sums behind lbm_tau1_stats). Work is queued on cuda_stream (NULL
 * = legacy default stream) and the call returns without waiting.
 * Errors: LBM_EINVAL (bad storage, NULL pointer, n < 1 or n larger than
 * LBM_TAU1_NOALLOC_MAX_NODES), LBM_ECUDA. The message of the calling
 * thread's last failure is in lbm_tau1_noalloc_last_error(). */
#define LBM_TAU1_NOALLOC_MAX_BLOCKS 1024
#define LBM_TAU1_NOALLOC_MAX_NODES (((int64_t)1) << 33)
lbm_status lbm_tau1_reduce_noalloc(int32_t storage, int64_t n, const void* drho, const void* ux, const void* uy,
                                   const void* uz, const float* inv_scale, const uint8_t* solid, const double* g,
                                   double* out, void* cuda_stream);
const char* lbm_tau1_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_TAU1_H */

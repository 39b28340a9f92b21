// Host-side launchers of the CUDA kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lbm {

// Tau1 step kernels (dense layout).
cudaError_t launch_tau1_simple(int q, int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_tau1_tiled(int q, int storage, int variant, const StepArgs& a, cudaStream_t s);
bool tau1_tiled_supported(int q, int storage, int64_t n);
int tau1_tiled_variants(int q, int storage);  // (row-pair + pair-position tile shapes) x z-chunk heights
int tau1_tile_shapes(int storage);            // tile shapes (the batched kernel's variants)
// Staged (TMA) form of the tiled kernel: same bits; for boxes with full tiles.
bool tau1_tiled_tma_ok(int q, int storage, int variant, const StepArgs& a);
cudaError_t launch_tau1_tiled_tma(int q, int storage, int variant, const StepArgs& a, cudaStream_t s);
// Tensor map of a state copy for the staged kernels: 3D {4 nx, ny, nz} values,
// box {4 (32 + 2 XOFF), box_rows, 1}.
cudaError_t encode_state_map(int storage, const void* base, int nx, int ny, int nz, int box_rows, CUtensorMap* map);
// Row-pair form (shuffle exchange within rows, shared memory across warp
// seams): same bits; for boxes with full tiles of its shape.
int tau1_rowpair_shapes(int storage);
bool tau1_rowpair_ok(int q, int storage, int shape, const StepArgs& a);
cudaError_t launch_tau1_rowpair(int q, int storage, int shape, int zchunk, const StepArgs& a, cudaStream_t s);
// Tile height (2W) of a row-pair shape (0 if none), and the row-pair kernel of
// a shape over a list of tile columns (indices b of the grid order: tile
// b % ntiles, z chunk b / ntiles, ntiles = (nx / 32) (ny / tile height)).
int tau1_rowpair_tile_height(int q, int storage, int shape);
cudaError_t launch_tau1_rowpair_list(int q, int storage, int shape, int zchunk, const StepArgs& a, const int* list,
                                     int count, cudaStream_t s);
// Self-test (selftest.cu): one warp waits, bounded, on an mbarrier phase
// that nothing completes and counts the timeout in *timeouts.
cudaError_t launch_selftest_timeout(unsigned int* timeouts, cudaStream_t s);

// Compact porous layout (compact.cu): tile columns of 32 x h x zchunk nodes,
// the unit of the row-pair variant (shape, zchunk) (variant v of
// [0, 2 tau1_rowpair_shapes): shape v mod R, zchunk 24 below R, else 32),
// numbered like that kernel's grid; fluid counts per tile column, and the
// fluid nodes of listed tile columns in row order at the given offsets.
struct CompactTiles {
    int shape, zchunk, h;
};
CompactTiles compact_tiles(int q, int storage, int variant);
int64_t compact_tile_columns(const CompactTiles& t, int nx, int ny, int nz);
int64_t compact_tile_nodes(const CompactTiles& t, int nx, int ny, int nz, int b);
cudaError_t launch_compact_count(const CompactTiles& t, int nx, int ny, int nz, const uint8_t* flags, int* counts,
                                 cudaStream_t s);
cudaError_t launch_compact_nodes(const CompactTiles& t, int nx, int ny, int nz, const uint8_t* flags, const int* tiles,
                                 const int* offsets, int ntiles, int* nodes, cudaStream_t s);
// Tau1 step of the listed box nodes (fluid), one thread per node, the
// neighbours gathered from the dense records (the dense kernels' values); the
// state copies hold n + 1 records, record n the solid sentinel written by
// launch_compact_sentinel (dscale: the 16-bit scales, or NULL).
cudaError_t launch_compact_sentinel(int storage, void* buf, int64_t n, const float* dscale, cudaStream_t s);
cudaError_t launch_tau1_list(int q, int storage, const StepArgs& a, const int* nodes, int64_t count, cudaStream_t s);

// D2Q9 (one plane): simple = one thread per node, else the y-marching warp
// kernel; same bits.
cudaError_t launch_tau1_2d(bool simple, int storage, const StepArgs& a, cudaStream_t s);
// Constant-density (Zou-He) faces of a non-periodic axis: overwrites the face
// nodes of a.post after a step from a.pre (q = 9, 19 or 27).
cudaError_t launch_zou_he(int q, int storage, const StepArgs& a, int axis, double rho_lo, double rho_hi,
                          cudaStream_t s);

// Sparse layout (fluid list + neighbour table). count: counts[0..nb) become
// the exclusive prefix sums of the fluid counts of the scan blocks and
// counts[nb] the total; build: idx (n ints) and pos (nf ints), then nbr
// ((q-1) nf ints). The step reads the list records of a.pre, writes a.post.
int sparse_scan_blocks(int64_t n);
cudaError_t launch_sparse_count(int64_t n, const uint8_t* flags, int* counts, cudaStream_t s);
cudaError_t launch_sparse_build(int q, int nx, int ny, int nz, const int periodic[3], const uint8_t* flags,
                                const int* offsets, int* idx, int* pos, int nf, int* nbr, cudaStream_t s);
cudaError_t launch_tau1_sparse(int q, int storage, const StepArgs& a, int nf, const int* nbr, cudaStream_t s);
cudaError_t launch_import_sparse(int storage, int nf, const double* const src[4], const int* pos, void* dst,
                                 const float scale[4], cudaStream_t s);
cudaError_t launch_export_sparse(int storage, int nf, const void* src, const int* pos, double* const dst[4],
                                 const float inv_scale[4], cudaStream_t s);

// Standard BGK (tau = 1, stored populations) comparison kernels. Populations:
// [q][n] in the storage type (FP32 or FP64). mask: one word per node of wall
// links (built by launch_bgk_mask from the node flags). init: populations from
// state records; moments: state records from the populations a step would gather.
bool bgk_supported(int q, int storage);
cudaError_t launch_bgk_mask(int q, const StepArgs& a, const uint8_t* flags, uint32_t* mask, cudaStream_t s);
cudaError_t launch_bgk_step(int q, int storage, const StepArgs& a, const void* fin, void* fout, const uint32_t* mask,
                            cudaStream_t s);
cudaError_t launch_bgk_moments(int q, int storage, const StepArgs& a, const void* fin, void* state,
                               const uint32_t* mask, cudaStream_t s);
cudaError_t launch_bgk_init(int q, int storage, const StepArgs& a, const void* state, void* fout, cudaStream_t s);

// 16-bit storage scales (device float[8]): re-chosen from the state's maxima
// by the headroom rule and applied to the state, all on the stream.
cudaError_t launch_rescale(int storage, int64_t n, void* state, const uint8_t* flags, float* dscale, float* partial,
                           float* ratio, double gmax, cudaStream_t s);
int rescale_scratch_floats(int64_t n);
void initial_scales(int storage, const double max_abs[4], double gmax, float scale[4]);

// Geometry preparation: node flags from the solid mask.
cudaError_t launch_build_flags(int q, int nx, int ny, int nz, const int periodic[3], const uint8_t* solid,
                               uint8_t* flags, cudaStream_t s);

// State records from FP64 arrays (drho, ux, uy, uz; src NULL = all zero);
// solid nodes get drho = NaN, u = 0.
cudaError_t launch_import_state(int storage, int64_t n, const double* const src[4], void* dst,
                                const uint8_t* flags, const float scale[4], cudaStream_t s);
// FP64 arrays from state records; solid nodes are reported as 0.
// inv_scale: host values (NULL = 1), replaced by the device array dinv[4] when dinv is not NULL.
cudaError_t launch_export_state(int storage, int64_t n, const void* src, double* const dst[4],
                                const uint8_t* flags, const float inv_scale[4], cudaStream_t s,
                                const float* dinv = nullptr);
// Largest |value| per field over the fluid nodes of FP64 arrays (16-bit scales).
cudaError_t launch_absmax_f64(int64_t n, const double* const src[4], const uint8_t* flags, double* out4,
                              double* scratch, int scratch_blocks, cudaStream_t s);

// FP64 reductions. partials holds reduce_blocks(n) * RED_FIELDS doubles; out
// receives RED_FIELDS doubles. flags NULL: every node is fluid (a fluid list). The state is either one array of records
// (aos = true, fields[0] the base) or four arrays of one field each.
enum { RED_NFLUID = 0, RED_DRHO, RED_PX, RED_PY, RED_PZ, RED_UMAX, RED_NONFINITE, RED_FIELDS = 8 };
int reduce_blocks(int64_t n);
// inv_scale: host values (NULL = 1), replaced by the device array dinv[4] when dinv is not NULL.
cudaError_t launch_reduce(int storage, bool aos, int64_t n, const void* const fields[4], const float inv_scale[4],
                          const uint8_t* flags, const double g[3], double* partials, double* out, cudaStream_t s,
                          const float* dinv = nullptr);

}  // namespace lbm

// Host-side launchers of the CUDA kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lbm {

// Tau1 step kernels (dense layout).
cudaError_t launch_tau1_simple(int q, int storage, const StepArgs& a, cudaStream_t s);
cudaError_t launch_tau1_tiled(int q, int storage, const StepArgs& a, cudaStream_t s);
bool tau1_tiled_supported(int q, int storage, int64_t n);
// Two-nodes-per-thread tiled kernel, packed f32x2 arithmetic (FP32/FP16/BF16 storage).
cudaError_t launch_tau1_pair(int q, int storage, int variant, const StepArgs& a, cudaStream_t s);
bool tau1_pair_supported(int q, int storage, int64_t n);
int tau1_pair_variants(int q);

// Geometry preparation: node flags from the solid mask.
cudaError_t launch_build_flags(int q, int nx, int ny, int nz, const int periodic[3], const uint8_t* solid,
                               uint8_t* flags, cudaStream_t s);

// State conversion between FP64 host/device arrays and the storage format.
// src/dst: drho, ux, uy, uz. Solid nodes are written as 0.
cudaError_t launch_import_fields(int storage, int64_t n, const double* const src[4], void* const dst[4],
                                 const uint8_t* flags, const float scale[4], cudaStream_t s);
cudaError_t launch_export_fields(int storage, int64_t n, const void* const src[4], double* const dst[4],
                                 const float inv_scale[4], cudaStream_t s);
// Largest |value| per field over the given FP64 arrays (for 16-bit scales).
cudaError_t launch_absmax_f64(int64_t n, const double* const src[4], const uint8_t* flags, double* out4,
                              double* scratch, int scratch_blocks, cudaStream_t s);

// FP64 reductions. partials holds reduce_blocks(n) * RED_FIELDS doubles; out
// receives RED_FIELDS doubles.
enum { RED_NFLUID = 0, RED_DRHO, RED_PX, RED_PY, RED_PZ, RED_UMAX, RED_NONFINITE, RED_FIELDS = 8 };
int reduce_blocks(int64_t n);
cudaError_t launch_reduce(int storage, int64_t n, const void* const fields[4], const float inv_scale[4],
                          const uint8_t* flags, const double g[3], double* partials, double* out, cudaStream_t s);

}  // namespace lbm

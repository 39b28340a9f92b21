// Shared device-side definitions of the CUDA path: node flags, storage
// formats of (drho, u), and the argument block of the step kernels.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lattice.cuh"

namespace lbm {

// Node flag byte (one per node, built from the solid mask at set_geometry).
enum : uint8_t {
    FLAG_SOLID = 1,      // node is solid: never updated, holds drho = 0, u = 0
    FLAG_WALL_LINK = 2,  // fluid node with at least one wall link x - c_k
};

enum : int { ST_F64 = 0, ST_F32 = 1, ST_F16S = 2, ST_BF16S = 3 };

// Storage of one field value. 16-bit formats hold value * scale (scale a
// power of two) and compute in FP32.
template <int ST> struct Storage;
template <> struct Storage<ST_F64> {
    using stype = double;
    using ctype = double;
    static constexpr int BYTES = 8;
    __device__ static __forceinline__ double load(const stype* p, int64_t i, float) { return __ldg(p + i); }
    __device__ static __forceinline__ void store(stype* p, int64_t i, double v, float) { p[i] = v; }
};
template <> struct Storage<ST_F32> {
    using stype = float;
    using ctype = float;
    static constexpr int BYTES = 4;
    __device__ static __forceinline__ float load(const stype* p, int64_t i, float) { return __ldg(p + i); }
    __device__ static __forceinline__ void store(stype* p, int64_t i, float v, float) { p[i] = v; }
};
template <> struct Storage<ST_F16S> {
    using stype = __half;
    using ctype = float;
    static constexpr int BYTES = 2;
    __device__ static __forceinline__ float load(const stype* p, int64_t i, float inv_scale)
    {
        return __half2float(__ldg(p + i)) * inv_scale;
    }
    __device__ static __forceinline__ void store(stype* p, int64_t i, float v, float scale)
    {
        p[i] = __float2half_rn(v * scale);
    }
};
template <> struct Storage<ST_BF16S> {
    using stype = __nv_bfloat16;
    using ctype = float;
    static constexpr int BYTES = 2;
    __device__ static __forceinline__ float load(const stype* p, int64_t i, float inv_scale)
    {
        return __bfloat162float(__ldg(p + i)) * inv_scale;
    }
    __device__ static __forceinline__ void store(stype* p, int64_t i, float v, float scale)
    {
        p[i] = __float2bfloat16_rn(v * scale);
    }
};

// Arguments of one Tau1 step on one dense box.
struct StepArgs {
    int nx, ny, nz;
    int periodic[3];
    double g[3];
    float gf[3];          // g rounded to FP32 (for FP32 arithmetic)
    const uint8_t* flags;
    const void* pre[4];   // drho, ux, uy, uz (read)
    void* post[4];        // drho, ux, uy, uz (written on fluid nodes only)
    float inv_scale[4];   // 16-bit storage: value = stored * inv_scale
    float scale[4];       // 16-bit storage: stored = value * scale
};

// Body force in the compute precision.
template <typename T> __device__ __forceinline__ T gcomp(const StepArgs& a, int i);
template <> __device__ __forceinline__ float gcomp<float>(const StepArgs& a, int i) { return a.gf[i]; }
template <> __device__ __forceinline__ double gcomp<double>(const StepArgs& a, int i) { return a.g[i]; }

// Reciprocal in the compute precision: FP64 correctly rounded; FP32 the
// hardware approximation (rcp.approx, at most 1 ulp from the exact value),
// used where rho = 1 + drho is near 1 and FP32 rounding dominates anyway.
__device__ __forceinline__ float recip(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

}  // namespace lbm

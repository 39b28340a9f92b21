// Shared device-side definitions of the CUDA path: node flags, the storage
// format of the state (drho, u), and the argument block of the step kernels.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lattice.cuh"

namespace lbm {

// Node flag byte (one per node, built from the solid mask at set_geometry).
// The step kernels do not read it (a solid node is marked in the state
// itself, below); geometry preparation, state I/O and reductions do.
enum : uint8_t {
    FLAG_SOLID = 1,      // node is solid: never updated
    FLAG_WALL_LINK = 2,  // fluid node with at least one wall link x - c_k
};

enum : int { ST_F64 = 0, ST_F32 = 1, ST_F16S = 2, ST_BF16S = 3 };

// State layout: one record per node, {drho, ux, uy, uz}, node index
// i = x + nx*(y + ny*z); 32 B (FP64), 16 B (FP32) or 8 B (16-bit formats).
// A thread that updates a node needs all four values of each source node, so
// one record is one vector load. Solid nodes hold drho = NaN and u = 0; the
// step kernels take a NaN drho as "solid" and never write solid nodes. The
// 16-bit formats hold value * scale (scale a power of two per field) and
// compute in FP32.
template <int ST> struct Storage;

template <> struct Storage<ST_F64> {
    using ctype = double;
    static constexpr int NODE_BYTES = 32;
    __device__ static __forceinline__ void load(const void* base, uint32_t i, const float*, double& d, double& ux,
                                                double& uy, double& uz)
    {
        const double2* p = static_cast<const double2*>(base) + 2 * (size_t)i;
        const double2 a = __ldg(p), b = __ldg(p + 1);
        d = a.x; ux = a.y; uy = b.x; uz = b.y;
    }
    __device__ static __forceinline__ void store(void* base, uint32_t i, double d, double ux, double uy, double uz,
                                                 const float*)
    {
        double2* p = static_cast<double2*>(base) + 2 * (size_t)i;
        p[0] = make_double2(d, ux);
        p[1] = make_double2(uy, uz);
    }
};

template <> struct Storage<ST_F32> {
    using ctype = float;
    static constexpr int NODE_BYTES = 16;
    __device__ static __forceinline__ void load(const void* base, uint32_t i, const float*, float& d, float& ux,
                                                float& uy, float& uz)
    {
        const float4 a = __ldg(static_cast<const float4*>(base) + i);
        d = a.x; ux = a.y; uy = a.z; uz = a.w;
    }
    __device__ static __forceinline__ void store(void* base, uint32_t i, float d, float ux, float uy, float uz,
                                                 const float*)
    {
        static_cast<float4*>(base)[i] = make_float4(d, ux, uy, uz);
    }
};

template <typename H> struct Storage16 {
    using ctype = float;
    static constexpr int NODE_BYTES = 8;
    __device__ static __forceinline__ float to_f(H h);
    __device__ static __forceinline__ H from_f(float f);
    __device__ static __forceinline__ void load(const void* base, uint32_t i, const float* inv, float& d, float& ux,
                                                float& uy, float& uz)
    {
        const uint2 w = __ldg(static_cast<const uint2*>(base) + i);
        const H* h = reinterpret_cast<const H*>(&w);
        d = to_f(h[0]) * inv[0];
        ux = to_f(h[1]) * inv[1];
        uy = to_f(h[2]) * inv[2];
        uz = to_f(h[3]) * inv[3];
    }
    __device__ static __forceinline__ void store(void* base, uint32_t i, float d, float ux, float uy, float uz,
                                                 const float* sc)
    {
        uint2 w;
        H* h = reinterpret_cast<H*>(&w);
        h[0] = from_f(d * sc[0]);
        h[1] = from_f(ux * sc[1]);
        h[2] = from_f(uy * sc[2]);
        h[3] = from_f(uz * sc[3]);
        static_cast<uint2*>(base)[i] = w;
    }
};
template <> __device__ __forceinline__ float Storage16<__half>::to_f(__half h) { return __half2float(h); }
template <> __device__ __forceinline__ __half Storage16<__half>::from_f(float f) { return __float2half_rn(f); }
template <> __device__ __forceinline__ float Storage16<__nv_bfloat16>::to_f(__nv_bfloat16 h)
{
    return __bfloat162float(h);
}
template <> __device__ __forceinline__ __nv_bfloat16 Storage16<__nv_bfloat16>::from_f(float f)
{
    return __float2bfloat16_rn(f);
}
template <> struct Storage<ST_F16S> : Storage16<__half> {};
template <> struct Storage<ST_BF16S> : Storage16<__nv_bfloat16> {};

inline int node_bytes(int st) { return st == ST_F64 ? 32 : (st == ST_F32 ? 16 : 8); }

// Arguments of one step on one dense box.
struct StepArgs {
    int nx, ny, nz;
    int periodic[3];
    double g[3];
    float gf[3];         // g rounded to FP32 (for FP32 arithmetic)
    const void* pre;     // state records read
    void* post;          // state records written (fluid nodes only)
    float inv_scale[4];  // 16-bit storage: value = stored * inv_scale
    float scale[4];      // 16-bit storage: stored = value * scale
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

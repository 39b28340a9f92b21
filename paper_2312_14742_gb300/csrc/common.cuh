// Shared device-side definitions of the CUDA path: node flags, the storage
// format of the state (drho, u), and the argument block of the step kernels.
#pragma once

#include <cstdint>
#include <type_traits>
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
    // one record at rec (any state space, e.g. shared memory)
    __device__ static __forceinline__ void load_at(const void* rec, const float*, double& d, double& ux, double& uy,
                                                   double& uz)
    {
        const double2* p = static_cast<const double2*>(rec);
        const double2 a = p[0], b = p[1];
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
    __device__ static __forceinline__ void load_at(const void* rec, const float*, float& d, float& ux, float& uy,
                                                   float& uz)
    {
        const float4 a = *static_cast<const float4*>(rec);
        d = a.x; ux = a.y; uy = a.z; uz = a.w;
    }
    __device__ static __forceinline__ void store(void* base, uint32_t i, float d, float ux, float uy, float uz,
                                                 const float*)
    {
        static_cast<float4*>(base)[i] = make_float4(d, ux, uy, uz);
    }
};

// Random bits for stochastic rounding: a counter-based hash of the node
// index and the step seed (an odd-multiplier / xor-shift mixer), so results
// are deterministic and the same in every kernel that stores the node.
__device__ __forceinline__ uint32_t sr_bits(uint32_t i, uint32_t seed)
{
    uint32_t h = i * 0x9E3779B1u + seed;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

// The 16-bit formats store value * S_f rounded stochastically (hardware
// cvt.rs: the result rounds up with probability equal to the fraction of
// the gap), so that updates smaller than half a unit in the last place still
// move the stored state in expectation instead of stalling it; loads are
// exact. Conversions outside the step kernels (import, re-scaling) use
// round-to-nearest.
template <typename H> struct Storage16 {
    using ctype = float;
    static constexpr int NODE_BYTES = 8;
    // BF16 has the FP32 exponent range and always keeps S_f = 1: no scaling
    static constexpr bool SCALED = !std::is_same<H, __nv_bfloat16>::value;
    __device__ static __forceinline__ float sc_mul(float v, float s) { return SCALED ? v * s : v; }
    __device__ static __forceinline__ float to_f(H h);
    __device__ static __forceinline__ H from_f(float f);
    __device__ static __forceinline__ uint32_t pack_sr(float lo, float hi, uint32_t r);
    __device__ static __forceinline__ void load(const void* base, uint32_t i, const float* inv, float& d, float& ux,
                                                float& uy, float& uz)
    {
        const uint2 w = __ldg(static_cast<const uint2*>(base) + i);
        decode(w, inv, d, ux, uy, uz);
    }
    __device__ static __forceinline__ void load_at(const void* rec, const float* inv, float& d, float& ux, float& uy,
                                                   float& uz)
    {
        decode(*static_cast<const uint2*>(rec), inv, d, ux, uy, uz);
    }
    __device__ static __forceinline__ void decode(uint2 w, const float* inv, float& d, float& ux, float& uy, float& uz)
    {
        const H* h = reinterpret_cast<const H*>(&w);
        d = sc_mul(to_f(h[0]), inv[0]);
        ux = sc_mul(to_f(h[1]), inv[1]);
        uy = sc_mul(to_f(h[2]), inv[2]);
        uz = sc_mul(to_f(h[3]), inv[3]);
    }
    // round to nearest
    __device__ static __forceinline__ void store(void* base, uint32_t i, float d, float ux, float uy, float uz,
                                                 const float* sc)
    {
        uint2 w;
        H* h = reinterpret_cast<H*>(&w);
        h[0] = from_f(sc_mul(d, sc[0]));
        h[1] = from_f(sc_mul(ux, sc[1]));
        h[2] = from_f(sc_mul(uy, sc[2]));
        h[3] = from_f(sc_mul(uz, sc[3]));
        static_cast<uint2*>(base)[i] = w;
    }
    // stochastic rounding with bits from sr_bits(i, seed)
    __device__ static __forceinline__ void store_sr(void* base, uint32_t i, float d, float ux, float uy, float uz,
                                                    const float* sc, uint32_t seed)
    {
        const uint32_t r = sr_bits(i, seed);
        uint2 w;
        w.x = pack_sr(sc_mul(d, sc[0]), sc_mul(ux, sc[1]), r);
        w.y = pack_sr(sc_mul(uy, sc[2]), sc_mul(uz, sc[3]), r * 0x85EBCA6Bu + 0x165667B1u);
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
// cvt.rs.*x2.f32 d, a, b: a goes to the upper half, b to the lower half.
template <> __device__ __forceinline__ uint32_t Storage16<__half>::pack_sr(float lo, float hi, uint32_t r)
{
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}
template <> __device__ __forceinline__ uint32_t Storage16<__nv_bfloat16>::pack_sr(float lo, float hi, uint32_t r)
{
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}
template <> struct Storage<ST_F16S> : Storage16<__half> {};
template <> struct Storage<ST_BF16S> : Storage16<__nv_bfloat16> {};

// Store of a step kernel: stochastic rounding for the 16-bit formats.
template <int ST, typename T>
__device__ __forceinline__ void step_store(void* base, uint32_t i, T d, T ux, T uy, T uz, const float* sc, uint32_t seed)
{
    if constexpr (ST == ST_F16S || ST == ST_BF16S) Storage<ST>::store_sr(base, i, d, ux, uy, uz, sc, seed);
    else Storage<ST>::store(base, i, d, ux, uy, uz, sc);
}

inline int node_bytes(int st) { return st == ST_F64 ? 32 : (st == ST_F32 ? 16 : 8); }

// Arguments of one step on one dense box.
struct StepArgs {
    int nx, ny, nz;
    int periodic[3];
    double g[3];
    float gf[3];         // g rounded to FP32 (for FP32 arithmetic)
    const void* pre;     // state records read
    void* post;          // state records written (fluid nodes only)
    float inv_scale[4];  // unused by the step kernels (see dscale)
    float scale[4];
    const float* dscale; // 16-bit storage: device float[8] = {S_f, 1/S_f}; stored = value * S_f
    uint32_t seed;       // stochastic-rounding seed of this step
    unsigned int* timeouts;  // device counter of staged-copy waits that ran out (staged kernels)
};

// Scales of the 16-bit formats, read once per thread from device memory.
// inv decodes the state read, s encodes the state written; one array
// {S, 1/S} serves both, or the read and written states have scales of their own.
struct Scales {
    float s[4], inv[4];
    __device__ __forceinline__ explicit Scales(const float* d) : Scales(d, d) {}
    __device__ __forceinline__ Scales(const float* pre, const float* post)
    {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            s[f] = post ? post[f] : 1.f;
            inv[f] = pre ? pre[4 + f] : 1.f;
        }
    }
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

// f2: two FP32 values (two lattice nodes handled by one thread) operated on
// with the packed f32x2 instructions of sm_100-class GPUs (one instruction
// issues both lanes). Each lane is an ordinary IEEE round-to-nearest FP32
// operation, so a lane gives bit for bit what the scalar code gives.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ explicit f2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit f2(double s) : v(make_float2((float)s, (float)s)) {}
    __device__ __forceinline__ explicit f2(int s) : v(make_float2((float)s, (float)s)) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit f2(float2 x) : v(x) {}
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
// a - b as b * (-1) + a: the product is exact, so this rounds like a - b
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { a = a + b; return a; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { a = a - b; return a; }

// rcp.approx per lane (no packed reciprocal exists)
__device__ __forceinline__ f2 recip(f2 x)
{
    float a, b;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(x.v.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(b) : "f"(x.v.y));
    return f2(a, b);
}

}  // namespace lbm

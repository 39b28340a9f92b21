// Two-lane arithmetic types: each thread of the tiled kernel updates two
// lattice nodes, lane A and lane B.
//
// f2: two FP32 values operated on with the packed f32x2 instructions of
// sm_100-class GPUs (one instruction issues both lanes). Each lane is an
// ordinary IEEE round-to-nearest FP32 operation, so a lane gives bit for bit
// what scalar code gives.
// d2: two FP64 values, one scalar instruction per lane.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct f2 {
    using elem = float;
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
// packed subtraction (sub.rn.f32x2): one IEEE rounding per lane like scalar
// a - b, and no register pair of -1 constants to keep or rebuild
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.v.x), "f"(a.v.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.v.x), "f"(b.v.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    f2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.v.x), "=f"(d.v.y) : "l"(rd));
    return d;
}
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

struct d2 {
    using elem = double;
    double2 v;
    __device__ __forceinline__ d2() {}
    __device__ __forceinline__ explicit d2(double s) : v(make_double2(s, s)) {}
    __device__ __forceinline__ explicit d2(float s) : v(make_double2((double)s, (double)s)) {}
    __device__ __forceinline__ explicit d2(int s) : v(make_double2((double)s, (double)s)) {}
    __device__ __forceinline__ d2(double a, double b) : v(make_double2(a, b)) {}
};

__device__ __forceinline__ d2 operator+(d2 a, d2 b) { return d2(__dadd_rn(a.v.x, b.v.x), __dadd_rn(a.v.y, b.v.y)); }
__device__ __forceinline__ d2 operator*(d2 a, d2 b) { return d2(__dmul_rn(a.v.x, b.v.x), __dmul_rn(a.v.y, b.v.y)); }
__device__ __forceinline__ d2 fma(d2 a, d2 b, d2 c) { return d2(::fma(a.v.x, b.v.x, c.v.x), ::fma(a.v.y, b.v.y, c.v.y)); }
__device__ __forceinline__ d2 operator-(d2 a, d2 b) { return d2(__dsub_rn(a.v.x, b.v.x), __dsub_rn(a.v.y, b.v.y)); }
__device__ __forceinline__ d2 operator-(d2 a) { return d2(-a.v.x, -a.v.y); }
__device__ __forceinline__ d2& operator+=(d2& a, d2 b) { a = a + b; return a; }
__device__ __forceinline__ d2& operator-=(d2& a, d2 b) { a = a - b; return a; }
__device__ __forceinline__ d2 recip(d2 x) { return d2(__drcp_rn(x.v.x), __drcp_rn(x.v.y)); }

template <typename E> struct Lanes;
template <> struct Lanes<float> { using type = f2; };
template <> struct Lanes<double> { using type = d2; };

}  // namespace lbm

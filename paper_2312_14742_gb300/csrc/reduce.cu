// Deterministic FP64 global reductions of one box's state.
//
// Pass 1: block b owns a fixed contiguous range of nodes; each thread sums a
// fixed strided subset, then a fixed shared-memory tree combines the block
// (warp shuffles for the last 32). Pass 2: one block combines the per-block
// partials in the same fixed way. The order of every addition depends only
// on n, so repeated calls give identical bits.
//
// Per fluid node: count, drho, physical velocity u + g/2 (three sums), the
// max of |u + g/2| (kept squared until the last pass), and a count of
// non-finite values.
#include "kernels.h"

namespace lbm {

static constexpr int RT = 256;  // threads per reduction block

int reduce_blocks(int64_t n)
{
    int64_t b = (n + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

struct Fields4 {
    const void* p[4];
};
struct Sc4r {
    float v[4];
};

__device__ __forceinline__ void combine(double* a, const double* b)
{
#pragma unroll
    for (int f = 0; f < RED_FIELDS; ++f) a[f] = (f == RED_UMAX) ? fmax(a[f], b[f]) : a[f] + b[f];
}

// Fixed-shape block reduction of RED_FIELDS doubles per thread; result in v of thread 0.
__device__ __forceinline__ void block_reduce(double* v, double (*sm)[RT])
{
#pragma unroll
    for (int f = 0; f < RED_FIELDS; ++f) sm[f][threadIdx.x] = v[f];
    __syncthreads();
    for (int w = RT / 2; w >= 32; w >>= 1) {
        if ((int)threadIdx.x < w) {
            double o[RED_FIELDS];
#pragma unroll
            for (int f = 0; f < RED_FIELDS; ++f) { v[f] = sm[f][threadIdx.x]; o[f] = sm[f][threadIdx.x + w]; }
            combine(v, o);
#pragma unroll
            for (int f = 0; f < RED_FIELDS; ++f) sm[f][threadIdx.x] = v[f];
        }
        __syncthreads();
    }
    if (threadIdx.x < 32) {
#pragma unroll
        for (int f = 0; f < RED_FIELDS; ++f) v[f] = sm[f][threadIdx.x];
        for (int off = 16; off > 0; off >>= 1) {
            double o[RED_FIELDS];
#pragma unroll
            for (int f = 0; f < RED_FIELDS; ++f) o[f] = __shfl_down_sync(0xffffffffu, v[f], off);
            combine(v, o);
        }
    }
}

// One field value of node i from an array of one field (plain storage
// element type of the format).
template <int ST> struct Plain;
template <> struct Plain<ST_F64> { __device__ static double get(const void* p, int64_t i, float) { return static_cast<const double*>(p)[i]; } };
template <> struct Plain<ST_F32> { __device__ static double get(const void* p, int64_t i, float) { return static_cast<const float*>(p)[i]; } };
template <> struct Plain<ST_F16S> {
    __device__ static double get(const void* p, int64_t i, float inv) { return __half2float(static_cast<const __half*>(p)[i]) * inv; }
};
template <> struct Plain<ST_BF16S> {
    __device__ static double get(const void* p, int64_t i, float inv)
    {
        return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]) * inv;
    }
};

template <int ST, bool AOS>
__global__ void __launch_bounds__(RT) reduce_pass1(int64_t n, Fields4 fl, Sc4r inv, const float* dinv,
                                                   const uint8_t* __restrict__ flags, double hgx, double hgy,
                                                   double hgz, double* __restrict__ partials)
{
    if (dinv)
#pragma unroll
        for (int f = 0; f < 4; ++f) inv.v[f] = dinv[f];
    using S = Storage<ST>;
    using T = typename S::ctype;
    __shared__ double sm[RED_FIELDS][RT];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per;
    const int64_t hi = lo + per < n ? lo + per : n;
    double v[RED_FIELDS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = lo + threadIdx.x; i < hi; i += RT) {
        if (flags && (flags[i] & FLAG_SOLID)) continue;
        double d, px, py, pz;
        if constexpr (AOS) {
            T v0, v1, v2, v3;
            S::load(fl.p[0], (uint32_t)i, inv.v, v0, v1, v2, v3);
            d = (double)v0;
            px = (double)v1 + hgx;
            py = (double)v2 + hgy;
            pz = (double)v3 + hgz;
        } else {
            d = Plain<ST>::get(fl.p[0], i, inv.v[0]);
            px = Plain<ST>::get(fl.p[1], i, inv.v[1]) + hgx;
            py = Plain<ST>::get(fl.p[2], i, inv.v[2]) + hgy;
            pz = Plain<ST>::get(fl.p[3], i, inv.v[3]) + hgz;
        }
        v[RED_NFLUID] += 1.0;
        v[RED_DRHO] += d;
        v[RED_PX] += px;
        v[RED_PY] += py;
        v[RED_PZ] += pz;
        // squared magnitude here; one square root of the maximum at the end
        // (sqrt is monotone and correctly rounded: the same value as the max of roots)
        const double m = px * px + py * py + pz * pz;
        if (isfinite(d) && isfinite(m)) v[RED_UMAX] = fmax(v[RED_UMAX], m);
        else v[RED_NONFINITE] += 1.0;
    }
    block_reduce(v, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int f = 0; f < RED_FIELDS; ++f) partials[(int64_t)blockIdx.x * RED_FIELDS + f] = v[f];
}

__global__ void __launch_bounds__(RT) reduce_pass2(int blocks, const double* __restrict__ partials, double* __restrict__ out)
{
    __shared__ double sm[RED_FIELDS][RT];
    double v[RED_FIELDS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < blocks; b += RT) combine(v, partials + (int64_t)b * RED_FIELDS);
    block_reduce(v, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int f = 0; f < RED_FIELDS; ++f) out[f] = f == RED_UMAX ? sqrt(v[f]) : v[f];
}

cudaError_t launch_reduce(int storage, bool aos, int64_t n, const void* const fields[4], const float inv_scale[4],
                          const uint8_t* flags, const double g[3], double* partials, double* out, cudaStream_t s,
                          const float* dinv)
{
    Fields4 f;
    Sc4r sc;
    for (int a = 0; a < 4; ++a) { f.p[a] = fields[a]; sc.v[a] = inv_scale ? inv_scale[a] : 1.f; }
    const int blocks = reduce_blocks(n);
    const double hx = 0.5 * g[0], hy = 0.5 * g[1], hz = 0.5 * g[2];
    switch (storage * 2 + (aos ? 1 : 0)) {
    case 2 * ST_F64: reduce_pass1<ST_F64, false><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    case 2 * ST_F64 + 1: reduce_pass1<ST_F64, true><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    case 2 * ST_F32: reduce_pass1<ST_F32, false><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    case 2 * ST_F32 + 1: reduce_pass1<ST_F32, true><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    case 2 * ST_F16S: reduce_pass1<ST_F16S, false><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    case 2 * ST_F16S + 1: reduce_pass1<ST_F16S, true><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    case 2 * ST_BF16S: reduce_pass1<ST_BF16S, false><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    case 2 * ST_BF16S + 1: reduce_pass1<ST_BF16S, true><<<blocks, RT, 0, s>>>(n, f, sc, dinv, flags, hx, hy, hz, partials); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_pass2<<<1, RT, 0, s>>>(blocks, partials, out);
    return cudaGetLastError();
}

}  // namespace lbm

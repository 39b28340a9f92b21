// Geometry preparation and state conversion kernels.
#include "kernels.h"
#include "static_for.cuh"

namespace lbm {

// flags[i] = FLAG_SOLID for solid nodes; FLAG_WALL_LINK for fluid nodes that
// have at least one wall link (a solid x - c_k, or one across a non-periodic
// face); 0 otherwise.
template <int Q, bool PLANE = false>
__global__ void build_flags_kernel(int nx, int ny, int nz, int px, int py, int pz, const uint8_t* __restrict__ solid,
                                   uint8_t* __restrict__ flags)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (solid[i]) { flags[i] = FLAG_SOLID; continue; }
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        bool wall = false;
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (PLANE && cvel(K, 2) != 0) return;  // D2Q9: the in-plane directions of D3Q19
            int sx = x - cvel(K, 0), sy = y - cvel(K, 1), sz = z - cvel(K, 2);
            bool out = false;
            if (sx < 0 || sx >= nx) { if (px) sx = sx < 0 ? sx + nx : sx - nx; else out = true; }
            if (sy < 0 || sy >= ny) { if (py) sy = sy < 0 ? sy + ny : sy - ny; else out = true; }
            if (sz < 0 || sz >= nz) { if (pz) sz = sz < 0 ? sz + nz : sz - nz; else out = true; }
            if (out || solid[(int64_t)sx + (int64_t)nx * ((int64_t)sy + (int64_t)ny * sz)]) wall = true;
        });
        flags[i] = wall ? FLAG_WALL_LINK : 0;
    }
}

static unsigned grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_build_flags(int q, int nx, int ny, int nz, const int periodic[3], const uint8_t* solid,
                               uint8_t* flags, cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny * nz;
    if (q == 9)
        build_flags_kernel<19, true><<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, periodic[0], periodic[1],
                                                                       periodic[2], solid, flags);
    else if (q == 19)
        build_flags_kernel<19><<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, periodic[0], periodic[1], periodic[2],
                                                                 solid, flags);
    else if (q == 27)
        build_flags_kernel<27><<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, periodic[0], periodic[1], periodic[2],
                                                                 solid, flags);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

struct F64x4 {
    const double* p[4];
};
struct D64x4 {
    double* p[4];
};
struct Sc4 {
    float v[4];
};

template <int ST>
__global__ void import_kernel(int64_t n, F64x4 src, void* dst, const uint8_t* __restrict__ flags, Sc4 scale)
{
    using S = Storage<ST>;
    using T = typename S::ctype;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v[4] = {T(0), T(0), T(0), T(0)};
        if (flags[i] & FLAG_SOLID) {
            v[0] = T(NAN);
        } else if (src.p[0]) {
#pragma unroll
            for (int f = 0; f < 4; ++f) v[f] = T(src.p[f][i]);
        }
        S::store(dst, (uint32_t)i, v[0], v[1], v[2], v[3], scale.v);
    }
}

template <int ST>
__global__ void export_kernel(int64_t n, const void* src, D64x4 dst, const uint8_t* __restrict__ flags, Sc4 inv,
                              const float* dinv)
{
    if (dinv)
#pragma unroll
        for (int f = 0; f < 4; ++f) inv.v[f] = dinv[f];
    using S = Storage<ST>;
    using T = typename S::ctype;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v[4];
        S::load(src, (uint32_t)i, inv.v, v[0], v[1], v[2], v[3]);
        const bool solid = flags[i] & FLAG_SOLID;
#pragma unroll
        for (int f = 0; f < 4; ++f)
            if (dst.p[f]) dst.p[f][i] = solid ? 0.0 : (double)v[f];
    }
}

cudaError_t launch_import_state(int storage, int64_t n, const double* const src[4], void* dst, const uint8_t* flags,
                                const float scale[4], cudaStream_t s)
{
    F64x4 a;
    Sc4 c;
    for (int f = 0; f < 4; ++f) { a.p[f] = src ? src[f] : nullptr; c.v[f] = scale[f]; }
    const unsigned g = grid_for(n, 256);
    switch (storage) {
    case ST_F64: import_kernel<ST_F64><<<g, 256, 0, s>>>(n, a, dst, flags, c); break;
    case ST_F32: import_kernel<ST_F32><<<g, 256, 0, s>>>(n, a, dst, flags, c); break;
    case ST_F16S: import_kernel<ST_F16S><<<g, 256, 0, s>>>(n, a, dst, flags, c); break;
    case ST_BF16S: import_kernel<ST_BF16S><<<g, 256, 0, s>>>(n, a, dst, flags, c); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_state(int storage, int64_t n, const void* src, double* const dst[4], const uint8_t* flags,
                                const float inv_scale[4], cudaStream_t s, const float* dinv)
{
    D64x4 b;
    Sc4 c;
    for (int f = 0; f < 4; ++f) { b.p[f] = dst[f]; c.v[f] = inv_scale ? inv_scale[f] : 1.f; }
    const unsigned g = grid_for(n, 256);
    switch (storage) {
    case ST_F64: export_kernel<ST_F64><<<g, 256, 0, s>>>(n, src, b, flags, c, dinv); break;
    case ST_F32: export_kernel<ST_F32><<<g, 256, 0, s>>>(n, src, b, flags, c, dinv); break;
    case ST_F16S: export_kernel<ST_F16S><<<g, 256, 0, s>>>(n, src, b, flags, c, dinv); break;
    case ST_BF16S: export_kernel<ST_BF16S><<<g, 256, 0, s>>>(n, src, b, flags, c, dinv); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Per-field max |value| over fluid nodes: one partial per block, then one block.
__global__ void absmax_pass1(int64_t n, F64x4 src, const uint8_t* __restrict__ flags, double* partial)
{
    __shared__ double sm[4][256];
    double m[4] = {0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flags[i] & FLAG_SOLID) continue;
#pragma unroll
        for (int f = 0; f < 4; ++f) m[f] = fmax(m[f], fabs(src.p[f][i]));
    }
    for (int f = 0; f < 4; ++f) sm[f][threadIdx.x] = m[f];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int f = 0; f < 4; ++f) sm[f][threadIdx.x] = fmax(sm[f][threadIdx.x], sm[f][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[blockIdx.x * 4 + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void absmax_pass2(int blocks, const double* partial, double* out)
{
    if (threadIdx.x < 4) {
        double m = 0;
        for (int b = 0; b < blocks; ++b) m = fmax(m, partial[b * 4 + threadIdx.x]);
        out[threadIdx.x] = m;
    }
}

cudaError_t launch_absmax_f64(int64_t n, const double* const src[4], const uint8_t* flags, double* out4,
                              double* scratch, int scratch_blocks, cudaStream_t s)
{
    F64x4 a;
    for (int f = 0; f < 4; ++f) a.p[f] = src[f];
    absmax_pass1<<<scratch_blocks, 256, 0, s>>>(n, a, flags, scratch);
    absmax_pass2<<<1, 32, 0, s>>>(scratch_blocks, scratch, out4);
    return cudaGetLastError();
}

}  // namespace lbm

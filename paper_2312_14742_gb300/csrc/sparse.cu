// Sparse layout: the state of the fluid nodes only, in a compact list, with a
// precomputed table of neighbour indices.
//
// The paper's kernels step every node of a dense box and skip solid chunks
// (Section 3.2); its outlook (Section 5) names indirect addressing of the
// fluid nodes for porous media with few fluid nodes. Here:
//   - fluid node i of the list is box node pos[i], in box order (x fastest),
//     numbered by an exclusive prefix sum of the fluid flags;
//   - nbr[(k-1) nf + i] is the list index of the source x - c_k of link k of
//     fluid node i (periodic axes wrapped), or -1 for a wall link (a solid
//     source or one across a non-periodic face);
//   - the step reads the own record, the index and the source record of each
//     link, and writes the own record: 2 (d+1) s + 4 (q-1) bytes per fluid
//     node from HBM when the source records come from cache.
// The per-link arithmetic and its order are those of the dense kernels
// (halfway bounce-back as fma(sigma, b, v); links c_z = +1, 0, -1, each in
// k order), so a sparse step gives the dense step's bits (FP32 and FP64).
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

constexpr int SCAN_T = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ bool fluid_at(const uint8_t* flags, int64_t n, int64_t i)
{
    return i < n && !(flags[i] & FLAG_SOLID);
}

// Block b: number of fluid nodes in [b SCAN_TILE, (b+1) SCAN_TILE).
__global__ void __launch_bounds__(SCAN_T) count_kernel(int64_t n, const uint8_t* __restrict__ flags, int* counts)
{
    __shared__ int sm[SCAN_T];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int c = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) c += fluid_at(flags, n, base + j) ? 1 : 0;
    sm[threadIdx.x] = c;
    __syncthreads();
    for (int w = SCAN_T / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = sm[0];
}

// Exclusive prefix sum of the block counts in place (one block, chunks of
// SCAN_T); total in counts[nblocks].
__global__ void __launch_bounds__(SCAN_T) scan_counts_kernel(int nblocks, int* counts)
{
    __shared__ int sm[SCAN_T];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nblocks; c0 += SCAN_T) {
        const int i = c0 + threadIdx.x;
        const int v = i < nblocks ? counts[i] : 0;
        sm[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < SCAN_T; off <<= 1) {  // inclusive Hillis-Steele scan
            const int t = (int)threadIdx.x >= off ? sm[threadIdx.x - off] : 0;
            __syncthreads();
            sm[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nblocks) counts[i] = carry + sm[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == SCAN_T - 1) carry += sm[SCAN_T - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[nblocks] = carry;
}

// List index of every box node (-1 for solid) and box node of every list entry.
__global__ void __launch_bounds__(SCAN_T) number_kernel(int64_t n, const uint8_t* __restrict__ flags,
                                                        const int* __restrict__ offsets, int* __restrict__ idx,
                                                        int* __restrict__ pos)
{
    __shared__ int sm[SCAN_T];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int c = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) c += fluid_at(flags, n, base + j) ? 1 : 0;
    sm[threadIdx.x] = c;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
        const int t = (int)threadIdx.x >= off ? sm[threadIdx.x - off] : 0;
        __syncthreads();
        sm[threadIdx.x] += t;
        __syncthreads();
    }
    int next = offsets[blockIdx.x] + sm[threadIdx.x] - c;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const int64_t i = base + j;
        if (i >= n) break;
        if (fluid_at(flags, n, i)) {
            idx[i] = next;
            pos[next] = (int)i;
            ++next;
        } else {
            idx[i] = -1;
        }
    }
}

template <int Q>
__global__ void __launch_bounds__(256) table_kernel(int nf, int nx, int ny, int nz, int px, int py, int pz,
                                                    const int* __restrict__ pos, const int* __restrict__ idx,
                                                    int* __restrict__ nbr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int64_t b = pos[i];
    const int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / ((int64_t)nx * ny));
    static_for<1, Q>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        int sx = x - cvel(K, 0), sy = y - cvel(K, 1), sz = z - cvel(K, 2);
        bool inside = true;
        if (sx < 0 || sx >= nx) { if (px) sx = sx < 0 ? sx + nx : sx - nx; else inside = false; }
        if (sy < 0 || sy >= ny) { if (py) sy = sy < 0 ? sy + ny : sy - ny; else inside = false; }
        if (sz < 0 || sz >= nz) { if (pz) sz = sz < 0 ? sz + nz : sz - nz; else inside = false; }
        const int j = inside ? idx[(int64_t)sx + (int64_t)nx * ((int64_t)sy + (int64_t)ny * sz)] : -1;
        nbr[(int64_t)(K - 1) * nf + i] = j;
    });
}

// One Tau1 step of the fluid list: one thread per fluid node.
template <int Q, int ST>
__global__ void __launch_bounds__(256) tau1_sparse_kernel(StepArgs a, int nf, const int* __restrict__ nbr)
{
    using S = Storage<ST>;
    using T = typename S::ctype;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const Scales sc(a.dscale);
    const T gx = gcomp<T>(a, 0), gy = gcomp<T>(a, 1), gz = gcomp<T>(a, 2);
    T d0, ux0, uy0, uz0;
    S::load(a.pre, (uint32_t)i, sc.inv, d0, ux0, uy0, uz0);
    const NodeMoments<T> own = node_moments<T>(d0, ux0, uy0, uz0, gx, gy, gz);
    NodeAcc<T, Weights<Q>::NCLASS> acc;
    acc.S[0] = own.A;

    auto link = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        const int j = __ldg(nbr + (int64_t)(K - 1) * nf + i);
        T v = T(0), sigma = T(1);
        if (j >= 0) {
            T d, ux, uy, uz;
            S::load(a.pre, (uint32_t)j, sc.inv, d, ux, uy, uz);
            const NodeMoments<T> m = node_moments<T>(d, ux, uy, uz, gx, gy, gz);
            v = feq_scaled(m.A, m.H, dir_dot<K, T>(m.Px, m.Py, m.Pz));
            sigma = T(0);
        }
        const T b = feq_scaled(own.A, own.H, -dir_dot<K, T>(own.Px, own.Py, own.Pz));
        acc.template add<Q, K>(fma(sigma, b, v));
    };
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 1) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 0) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == -1) link(kc); });

    T d, ux, uy, uz;
    node_finish<Q, T>(acc, d, ux, uy, uz);
    step_store<ST>(a.post, (uint32_t)i, d, ux, uy, uz, sc.s, a.seed);
}

struct F64x4s {
    const double* p[4];
};
struct D64x4s {
    double* p[4];
};
struct Sc4s {
    float v[4];
};

// records of the list from dense FP64 arrays (src NULL: all zero)
template <int ST>
__global__ void import_sparse_kernel(int nf, F64x4s src, const int* __restrict__ pos, void* dst, Sc4s scale)
{
    using T = typename Storage<ST>::ctype;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    T v[4] = {T(0), T(0), T(0), T(0)};
    if (src.p[0]) {
        const int64_t b = pos[i];
#pragma unroll
        for (int f = 0; f < 4; ++f) v[f] = T(src.p[f][b]);
    }
    Storage<ST>::store(dst, (uint32_t)i, v[0], v[1], v[2], v[3], scale.v);
}

// dense FP64 arrays from the list (the solid nodes were zeroed before)
template <int ST>
__global__ void export_sparse_kernel(int nf, const void* src, const int* __restrict__ pos, D64x4s dst, Sc4s inv)
{
    using T = typename Storage<ST>::ctype;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    T v[4];
    Storage<ST>::load(src, (uint32_t)i, inv.v, v[0], v[1], v[2], v[3]);
    const int64_t b = pos[i];
#pragma unroll
    for (int f = 0; f < 4; ++f)
        if (dst.p[f]) dst.p[f][b] = (double)v[f];
}

template <int Q>
cudaError_t launch_step_q(int storage, const StepArgs& a, int nf, const int* nbr, cudaStream_t s)
{
    const unsigned g = (unsigned)((nf + 255) / 256);
    switch (storage) {
    case ST_F64: tau1_sparse_kernel<Q, ST_F64><<<g, 256, 0, s>>>(a, nf, nbr); break;
    case ST_F32: tau1_sparse_kernel<Q, ST_F32><<<g, 256, 0, s>>>(a, nf, nbr); break;
    case ST_F16S: tau1_sparse_kernel<Q, ST_F16S><<<g, 256, 0, s>>>(a, nf, nbr); break;
    case ST_BF16S: tau1_sparse_kernel<Q, ST_BF16S><<<g, 256, 0, s>>>(a, nf, nbr); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int sparse_scan_blocks(int64_t n) { return (int)((n + SCAN_TILE - 1) / SCAN_TILE); }

cudaError_t launch_sparse_count(int64_t n, const uint8_t* flags, int* counts, cudaStream_t s)
{
    const int nb = sparse_scan_blocks(n);
    count_kernel<<<nb, SCAN_T, 0, s>>>(n, flags, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scan_counts_kernel<<<1, SCAN_T, 0, s>>>(nb, counts);
    return cudaGetLastError();
}

cudaError_t launch_sparse_build(int q, int nx, int ny, int nz, const int periodic[3], const uint8_t* flags,
                                const int* offsets, int* idx, int* pos, int nf, int* nbr, cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny * nz;
    number_kernel<<<sparse_scan_blocks(n), SCAN_T, 0, s>>>(n, flags, offsets, idx, pos);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nf == 0) return e;
    const unsigned g = (unsigned)((nf + 255) / 256);
    if (q == 19)
        table_kernel<19><<<g, 256, 0, s>>>(nf, nx, ny, nz, periodic[0], periodic[1], periodic[2], pos, idx, nbr);
    else
        table_kernel<27><<<g, 256, 0, s>>>(nf, nx, ny, nz, periodic[0], periodic[1], periodic[2], pos, idx, nbr);
    return cudaGetLastError();
}

cudaError_t launch_tau1_sparse(int q, int storage, const StepArgs& a, int nf, const int* nbr, cudaStream_t s)
{
    if (nf == 0) return cudaSuccess;
    return q == 19 ? launch_step_q<19>(storage, a, nf, nbr, s) : launch_step_q<27>(storage, a, nf, nbr, s);
}

cudaError_t launch_import_sparse(int storage, int nf, const double* const src[4], const int* pos, void* dst,
                                 const float scale[4], cudaStream_t s)
{
    if (nf == 0) return cudaSuccess;
    F64x4s a;
    Sc4s c;
    for (int f = 0; f < 4; ++f) { a.p[f] = src ? src[f] : nullptr; c.v[f] = scale[f]; }
    const unsigned g = (unsigned)((nf + 255) / 256);
    switch (storage) {
    case ST_F64: import_sparse_kernel<ST_F64><<<g, 256, 0, s>>>(nf, a, pos, dst, c); break;
    case ST_F32: import_sparse_kernel<ST_F32><<<g, 256, 0, s>>>(nf, a, pos, dst, c); break;
    case ST_F16S: import_sparse_kernel<ST_F16S><<<g, 256, 0, s>>>(nf, a, pos, dst, c); break;
    case ST_BF16S: import_sparse_kernel<ST_BF16S><<<g, 256, 0, s>>>(nf, a, pos, dst, c); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_sparse(int storage, int nf, const void* src, const int* pos, double* const dst[4],
                                 const float inv_scale[4], cudaStream_t s)
{
    if (nf == 0) return cudaSuccess;
    D64x4s b;
    Sc4s c;
    for (int f = 0; f < 4; ++f) { b.p[f] = dst[f]; c.v[f] = inv_scale[f]; }
    const unsigned g = (unsigned)((nf + 255) / 256);
    switch (storage) {
    case ST_F64: export_sparse_kernel<ST_F64><<<g, 256, 0, s>>>(nf, src, pos, b, c); break;
    case ST_F32: export_sparse_kernel<ST_F32><<<g, 256, 0, s>>>(nf, src, pos, b, c); break;
    case ST_F16S: export_sparse_kernel<ST_F16S><<<g, 256, 0, s>>>(nf, src, pos, b, c); break;
    case ST_BF16S: export_sparse_kernel<ST_BF16S><<<g, 256, 0, s>>>(nf, src, pos, b, c); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm

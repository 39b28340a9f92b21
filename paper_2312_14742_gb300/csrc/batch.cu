// Batched persistent Tau1 step: many dense boxes of different sizes advance
// one step in one launch.
//
// The work of a step is the list of tile columns of every live box (box-major,
// each box chunk-major as in the single-box kernel). Columns are `chunk`
// planes high; the host lowers the chunk (32 down to 4 planes) when few boxes
// are live, so that a step spreads over the SMs and its latency, one column,
// stays short. A node's result does not depend on the chunk. A grid of (SMs x resident
// blocks) works through the list: each block takes its first item by its
// index and then the next unclaimed one (an atomic counter), so blocks that
// drew small items (partial tiles or chunks, small boxes) take more of them.
// Each item is one tile_column() call with that box's arguments, read from the
// device table. Everything that changes from step to
// step lives in the table on the device: which copy holds a box's current
// state, its step count (the stochastic-rounding seed), its 16-bit scales.
// Boxes whose tiles are all full are stepped by a staged (TMA) instance of
// the kernel (the row-pair tile column for variant 0, rowpair.cuh) through
// their own tensor maps (one per state copy, in device
// memory; the stage mbarriers are set up once per launch and their phases run
// on from item to item), the others by a register instance: two work tables,
// one launch each per step. A launch therefore has the same arguments every
// step, and K steps can be captured once in a CUDA graph and replayed while
// boxes come and go (the host edits the table between replays). The two
// tables hold different boxes, so the graph holds them as two independent
// chains of K launches that run side by side.
//
// The last block to finish (an atomic count, no waiting) closes the step for
// every live box: swaps its copies, counts the step and, for FP16 storage,
// picks the scale of the next written copy by the headroom rule from the
// maxima that the blocks gathered while storing. The state written and the
// scales chosen depend only on the box's own state and step count, so a box
// gives the same bits alone and in any mix.
#include "batch.h"
#include "rowpair.cuh"
#include "tile_column.cuh"

namespace lbm {

namespace {

using namespace tile;

__device__ __forceinline__ uint32_t step_seed(int64_t step) { return (uint32_t)(step + 1) * 0x9E3779B9u; }

// Headroom rule of the 16-bit scales (FP16): reference magnitude
// r = max(m_f, max_f' m_f' / 16, 64 |g|_max); S = 2^(12 - e(r)) when
// m_f S > 2^13 or r S < 2^9.
__device__ float decide_scale(const float m[4], int f, float s_old, float gfloor)
{
    const float mall = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
    const float ref = fmaxf(fmaxf(m[f], 0.0625f * mall), gfloor);
    if (!(ref > 0.f) || !isfinite(mall)) return s_old;
    if (m[f] * s_old <= 8192.f && ref * s_old >= 512.f) return s_old;
    int e;
    frexpf(ref, &e);
    e = 12 - e;
    e = e > 100 ? 100 : (e < -100 ? -100 : e);
    return ldexpf(1.f, e);
}

__device__ void finish_box(BatchDomain& R, int storage)
{
    const uint32_t c = R.cur;
    const int64_t step = R.step + 1;
    if (storage == ST_F16S || storage == ST_BF16S) {
        // buf[c ^ 1] was just written with scale[c ^ 1]; the next step writes buf[c]
        const bool check = storage == ST_F16S && step % BATCH_RESCALE_EVERY == 0;
        float m[4] = {0.f, 0.f, 0.f, 0.f};
        if (check)
#pragma unroll
            for (int f = 0; f < 4; ++f) m[f] = __uint_as_float(atomicExch(&R.amax[f], 0u));
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float s = check ? decide_scale(m, f, R.scale[c ^ 1][f], R.gfloor) : R.scale[c ^ 1][f];
            R.scale[c][f] = s;
            R.scale[c][4 + f] = 1.f / s;
        }
    }
    R.cur = c ^ 1;
    R.step = step;
}

// RP: the staged instance steps its items with the row-pair tile column
// (rowpair_column, tile 32 x 2H: the same tiles, tensor maps and bits).
template <int Q, int ST, int H, int MINB, bool TMA, bool RP>
__global__ void __launch_bounds__(32 * H, MINB) tau1_batch_kernel(BatchTable* T)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // the row-pair stage buffers want 128-byte alignment
    unsigned char* smem_raw = RP ? smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u) : smem_dyn;
    __shared__ int last;
    // FP16 only (BF16 keeps S = 1): maxima of the stored values, needed on the
    // step before each scale check
    constexpr bool AMAX = ST == ST_F16S;
    const int nitems = T->nitems, ndom = T->ndom, chunk = T->chunk;
    const int* __restrict__ begin = T->item_begin;
    // visible after the first item's barrier
    if constexpr (RP) rp::rp_stage_init<Q, ST, H>(smem_raw);
    else if constexpr (TMA) stage_init<Q, ST, H>(smem_raw);
    uint32_t phase = 0;
    __shared__ int next_item;
    // each block takes its first item by its index, then the next free one
    // (items differ in size: partial tiles, partial chunks, several boxes)
    for (int it = blockIdx.x; it < nitems;) {
        // box of this item: the last d with begin[d] <= it
        int lo = 0, hi = ndom - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (begin[mid] <= it) lo = mid;
            else hi = mid - 1;
        }
        const int slot = T->live[lo];
        BatchDomain& R = T->dom[slot];
        const int local = it - begin[lo];
        StepArgs a = R.a;
        const uint32_t c = R.cur;
        a.pre = R.buf[c];
        a.post = R.buf[c ^ 1];
        a.seed = step_seed(R.step);
        const Scales sc(AMAX ? R.scale[c] : nullptr, AMAX ? R.scale[c ^ 1] : nullptr);
        const int tile = local % R.ntiles;
        const int z0 = (local / R.ntiles) * chunk;
        const int z1 = min(a.nz, z0 + chunk);
        const int x0 = (tile % R.ntx) * 32, y0 = (tile / R.ntx) * (2 * H);
        float amax[4] = {0.f, 0.f, 0.f, 0.f};
        __syncthreads();  // the previous item's last shared-memory reads are done
        if constexpr (RP)
            rp::rowpair_column<Q, ST, H, AMAX>(a, sc, x0, y0, z0, z1, smem_raw, amax, T->maps + 2 * slot + c, &phase);
        else if constexpr (TMA)
            tile_column<Q, ST, H, AMAX, true>(a, sc, x0, y0, z0, z1, smem_raw, amax, T->maps + 2 * slot + c, &phase);
        else
            tile_column<Q, ST, H, AMAX, false>(a, sc, x0, y0, z0, z1, smem_raw, amax);
        if (AMAX && (R.step + 1) % BATCH_RESCALE_EVERY == 0) {
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                float m = amax[f];
                for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                // non-negative floats order like their bit patterns
                if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&R.amax[f], __float_as_uint(m));
            }
        }
        if (threadIdx.x == 0) next_item = (int)gridDim.x + (int)atomicAdd(&T->next, 1u);
        __syncthreads();
        it = next_item;
    }
    // close the step: the last block to arrive updates every live box
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&T->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int d = threadIdx.x; d < ndom; d += blockDim.x) finish_box(T->dom[T->live[d]], ST);
    if (threadIdx.x == 0) {
        T->done = 0;
        T->next = 0;
    }
}

template <int Q, int ST, int V, bool TMA>
struct BatchKernel {
    using E = typename Storage<ST>::ctype;
    static constexpr int H = Shape<Q, E, V>::H;
    using C = TCfg<Q, 32, H, E>;
    // variant 0 of the staged instance: the row-pair form of the same tile, at
    // the single-box row-pair kernel's block count (a few bytes of spills in
    // FP32 at 4 blocks: measured faster on serving mixes than 3 blocks)
    static constexpr bool RP = TMA && V == 0 && rp::RShape<Q, E, 0>::W == H;
    static constexpr int MINB = RP ? rp::RShape<Q, E, 0>::MINB : Shape<Q, E, V>::MINB;
    static constexpr size_t SMEM = RP ? rp::rowpair_smem<Q, ST, H>() + 128 : tile_smem<Q, ST, H, TMA>();
    static_assert(SMEM <= 227 * 1024, "shared memory of one block");
    static constexpr auto fn() { return tau1_batch_kernel<Q, ST, H, MINB, TMA, RP>; }
    static cudaError_t prepare(int& grid, int& tile_h)
    {
        auto kern = fn();
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, SMEM)) != cudaSuccess)
            return e;
        grid = sms * (per_sm > 0 ? per_sm : 1);
        tile_h = 2 * H;
        return cudaSuccess;
    }
    static cudaError_t launch(BatchTable* T, int grid, cudaStream_t s)
    {
        fn()<<<grid, C::NT, SMEM, s>>>(T);
        return cudaGetLastError();
    }
};

template <int Q, int ST, bool TMA>
cudaError_t dispatch_v(int variant, bool prep, BatchTable* T, int& grid, int& tile_h, cudaStream_t s)
{
    auto go = [&](auto k) {
        using K = decltype(k);
        return prep ? K::prepare(grid, tile_h) : K::launch(T, grid, s);
    };
    if constexpr (ST == ST_F64) {
        return variant == 0 ? go(BatchKernel<Q, ST, 0, TMA>{}) : cudaErrorInvalidValue;
    } else {
        switch (variant) {
        case 0: return go(BatchKernel<Q, ST, 0, TMA>{});
        case 1: return go(BatchKernel<Q, ST, 1, TMA>{});
        case 2: return go(BatchKernel<Q, ST, 2, TMA>{});
        case 3: return go(BatchKernel<Q, ST, 3, TMA>{});
        default: return cudaErrorInvalidValue;
        }
    }
}

template <bool TMA>
cudaError_t dispatch(int q, int storage, int variant, bool prep, BatchTable* T, int& grid, int& tile_h,
                     cudaStream_t s)
{
    switch (q * 10 + storage) {
    case 190 + ST_F64: return dispatch_v<19, ST_F64, TMA>(variant, prep, T, grid, tile_h, s);
    case 190 + ST_F32: return dispatch_v<19, ST_F32, TMA>(variant, prep, T, grid, tile_h, s);
    case 190 + ST_F16S: return dispatch_v<19, ST_F16S, TMA>(variant, prep, T, grid, tile_h, s);
    case 190 + ST_BF16S: return dispatch_v<19, ST_BF16S, TMA>(variant, prep, T, grid, tile_h, s);
    case 270 + ST_F64: return dispatch_v<27, ST_F64, TMA>(variant, prep, T, grid, tile_h, s);
    case 270 + ST_F32: return dispatch_v<27, ST_F32, TMA>(variant, prep, T, grid, tile_h, s);
    case 270 + ST_F16S: return dispatch_v<27, ST_F16S, TMA>(variant, prep, T, grid, tile_h, s);
    case 270 + ST_BF16S: return dispatch_v<27, ST_BF16S, TMA>(variant, prep, T, grid, tile_h, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t batch_prepare(int q, int storage, int variant, bool tma, int* grid, int* tile_h)
{
    int g = 0, th = 0;
    cudaError_t e = tma ? dispatch<true>(q, storage, variant, true, nullptr, g, th, nullptr)
                        : dispatch<false>(q, storage, variant, true, nullptr, g, th, nullptr);
    *grid = g;
    *tile_h = th;
    return e;
}

cudaError_t launch_tau1_batch(int q, int storage, int variant, bool tma, BatchTable* T, int grid, cudaStream_t s)
{
    int th = 0;
    return tma ? dispatch<true>(q, storage, variant, false, T, grid, th, s)
               : dispatch<false>(q, storage, variant, false, T, grid, th, s);
}

}  // namespace lbm

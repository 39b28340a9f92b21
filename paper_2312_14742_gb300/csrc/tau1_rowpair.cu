// Row-pair Tau1 step kernel for one dense box whose tiles are all full (nx a
// multiple of 32, ny of the tile height 2W): one block of W warps per tile
// column (a 32 x 2W tile of the x-y plane, a z-chunk of planes), grid ordered
// chunk-major so that the tiles of a chunk run side by side and their halo
// reads hit L2. The update itself is rowpair_column() (rowpair.cuh); it gives
// the same bits as the other step kernels of this library.
#include <cudaTypedefs.h>

#include "rowpair.cuh"

namespace lbm {

namespace {

using namespace rp;

template <int Q, int ST, int W, int MINB>
__global__ void __launch_bounds__(32 * W, MINB)
    tau1_rowpair_kernel(StepArgs a, int ntx, int ntiles, int chunk, const __grid_constant__ CUtensorMap tmap,
                        const int* __restrict__ list)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // stage buffers of the tensor copies want 128-byte alignment
    unsigned char* smem = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    // the tile columns of the whole box in grid order, or those of a list
    const int b = list ? list[blockIdx.x] : (int)blockIdx.x;
    const int tile = b % ntiles;
    const int z0 = (b / ntiles) * chunk;
    const int z1 = min(a.nz, z0 + chunk);
    const int x0 = (tile % ntx) * 32, y0 = (tile / ntx) * (2 * W);
    const Scales sc(a.dscale);
    float amax[4];
    rp_stage_init<Q, ST, W>(smem);
    __syncthreads();
    uint32_t phase = 0;
    rowpair_column<Q, ST, W, false>(a, sc, x0, y0, z0, z1, smem, amax, &tmap, &phase);
}

template <int Q, int ST, int V>
cudaError_t launch_t(const StepArgs& a, int zchunk, cudaStream_t s, const int* list = nullptr, int count = 0)
{
    using E = typename Storage<ST>::ctype;
    constexpr int W = RShape<Q, E, V>::W;
    constexpr size_t SMEM = rowpair_smem<Q, ST, W>() + 128;
    static_assert(SMEM <= 227 * 1024, "shared memory of one block");
    auto kern = tau1_rowpair_kernel<Q, ST, W, RShape<Q, E, V>::MINB>;
    // the attribute is per device; setting it on every launch is cheap
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    e = encode_state_map(ST, a.pre, a.nx, a.ny, a.nz, 2 * W + 2, &map);
    if (e != cudaSuccess) return e;
    const int ntx = a.nx / 32;
    const int ntiles = ntx * (a.ny / (2 * W));
    const int chunk = a.nz < zchunk ? a.nz : zchunk;
    const int nchunks = (a.nz + chunk - 1) / chunk;
    const long long blocks = list ? (long long)count : (long long)ntiles * nchunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (blocks == 0) return cudaSuccess;
    kern<<<(unsigned)blocks, 32 * W, SMEM, s>>>(a, ntx, ntiles, chunk, map, list);
    return cudaGetLastError();
}

template <int Q, int ST>
cudaError_t launch_s(int shape, int zchunk, const StepArgs& a, cudaStream_t s, const int* list = nullptr,
                     int count = 0)
{
    if constexpr (ST == ST_F64) {
        return shape == 0 ? launch_t<Q, ST, 0>(a, zchunk, s, list, count) : cudaErrorInvalidValue;
    } else {
        switch (shape) {
        case 0: return launch_t<Q, ST, 0>(a, zchunk, s, list, count);
        case 1: return launch_t<Q, ST, 1>(a, zchunk, s, list, count);
        case 2: return launch_t<Q, ST, 2>(a, zchunk, s, list, count);
        case 3: return launch_t<Q, ST, 3>(a, zchunk, s, list, count);
        default: return cudaErrorInvalidValue;
        }
    }
}

int shape_w(int q, int storage, int shape)
{
    if (storage == ST_F64) return shape == 0 ? RShape<19, double, 0>::W : 0;
    if (shape < 0 || shape >= RSHAPES) return 0;
    constexpr int w19[4] = {RShape<19, float, 0>::W, RShape<19, float, 1>::W, RShape<19, float, 2>::W,
                            RShape<19, float, 3>::W};
    constexpr int w27[4] = {RShape<27, float, 0>::W, RShape<27, float, 1>::W, RShape<27, float, 2>::W,
                            RShape<27, float, 3>::W};
    return q == 19 ? w19[shape] : w27[shape];
}

}  // namespace

int tau1_rowpair_shapes(int storage) { return storage == ST_F64 ? 1 : RSHAPES; }

bool tau1_rowpair_ok(int q, int storage, int shape, const StepArgs& a)
{
    const int w = shape_w(q, storage, shape);
    if (w == 0 || a.nx % 32 != 0 || a.ny % (2 * w) != 0) return false;
    if (!a.timeouts) return false;
    // a box row of 16-bit records starts at a multiple of 16 bytes only if nx is even
    if ((reinterpret_cast<uintptr_t>(a.pre) & 15) != 0) return false;
    CUtensorMap probe;
    return encode_state_map(storage, a.pre, a.nx, a.ny, a.nz, 2 * w + 2, &probe) == cudaSuccess;
}

int tau1_rowpair_tile_height(int q, int storage, int shape) { return 2 * shape_w(q, storage, shape); }

cudaError_t launch_tau1_rowpair_list(int q, int storage, int shape, int zchunk, const StepArgs& a, const int* list,
                                     int count, cudaStream_t s)
{
    if (!list) return cudaErrorInvalidValue;
    switch (q * 10 + storage) {
    case 190 + ST_F64: return launch_s<19, ST_F64>(shape, zchunk, a, s, list, count);
    case 190 + ST_F32: return launch_s<19, ST_F32>(shape, zchunk, a, s, list, count);
    case 190 + ST_F16S: return launch_s<19, ST_F16S>(shape, zchunk, a, s, list, count);
    case 190 + ST_BF16S: return launch_s<19, ST_BF16S>(shape, zchunk, a, s, list, count);
    case 270 + ST_F64: return launch_s<27, ST_F64>(shape, zchunk, a, s, list, count);
    case 270 + ST_F32: return launch_s<27, ST_F32>(shape, zchunk, a, s, list, count);
    case 270 + ST_F16S: return launch_s<27, ST_F16S>(shape, zchunk, a, s, list, count);
    case 270 + ST_BF16S: return launch_s<27, ST_BF16S>(shape, zchunk, a, s, list, count);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tau1_rowpair(int q, int storage, int shape, int zchunk, const StepArgs& a, cudaStream_t s)
{
    switch (q * 10 + storage) {
    case 190 + ST_F64: return launch_s<19, ST_F64>(shape, zchunk, a, s);
    case 190 + ST_F32: return launch_s<19, ST_F32>(shape, zchunk, a, s);
    case 190 + ST_F16S: return launch_s<19, ST_F16S>(shape, zchunk, a, s);
    case 190 + ST_BF16S: return launch_s<19, ST_BF16S>(shape, zchunk, a, s);
    case 270 + ST_F64: return launch_s<27, ST_F64>(shape, zchunk, a, s);
    case 270 + ST_F32: return launch_s<27, ST_F32>(shape, zchunk, a, s);
    case 270 + ST_F16S: return launch_s<27, ST_F16S>(shape, zchunk, a, s);
    case 270 + ST_BF16S: return launch_s<27, ST_BF16S>(shape, zchunk, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

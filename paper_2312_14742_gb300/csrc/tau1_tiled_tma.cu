// Staged tiled Tau1 step kernel: the tiled kernel with each plane's box of
// raw records (tile plus one-node halo ring) copied into shared memory by the
// tensor unit (cp.async.bulk.tensor), two planes ahead of its use, instead of
// per-thread global loads held in registers across the plane barrier.
//
// It serves boxes whose tiles are all full (nx a multiple of 32, ny of the
// tile height), so every tile lies inside the box; halo nodes outside it come
// back zero-filled from the copy and are read from global memory (periodic
// images, which the copy cannot wrap) or are walls. Ragged boxes use the
// register form: handling a ragged last tile here, even behind a block-uniform
// branch, cost 6% on full tiles.
// The state is viewed as a 3D array of 4 nx x ny x nz values (one record is
// 4 values), so that a box row of 34 records starts at an element coordinate
// that is a multiple of 4 values: a multiple of 16 bytes for every format.
#include <cudaTypedefs.h>

#include "tile_column.cuh"

namespace lbm {

namespace {

using namespace tile;

template <int Q, int ST, int H, int MINB>
__global__ void __launch_bounds__(32 * H, MINB)
    tau1_tiled_tma_kernel(StepArgs a, int ntx, int ntiles, int chunk, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tile = blockIdx.x % ntiles;
    const int z0 = (blockIdx.x / ntiles) * chunk;
    const int z1 = min(a.nz, z0 + chunk);
    const int x0 = (tile % ntx) * 32, y0 = (tile / ntx) * (2 * H);
    const Scales sc(a.dscale);
    float amax[4];
    stage_init<Q, ST, H>(smem_raw);
    __syncthreads();
    uint32_t phase = 0;
    tile_column<Q, ST, H, false, true>(a, sc, x0, y0, z0, z1, smem_raw, amax, &tmap, &phase);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of the state read by a step: 3D, dims {4 nx, ny, nz} values,
// box {4 * 34, 2H + 2, 1}.
template <int ST> cudaError_t encode_state(CUtensorMap* map, const StepArgs& a, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    using SC = StageCfg<ST, 1>;
    constexpr int es = SC::REC / 4;
    const CUtensorMapDataType dt = ST == ST_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : ST == ST_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                  : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[3] = {(cuuint64_t)4 * a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)4 * es * a.nx, (cuuint64_t)4 * es * a.nx * a.ny};
    const cuuint32_t box[3] = {(cuuint32_t)SC::BOX_X, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, dt, 3, const_cast<void*>(a.pre), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int ST> cudaError_t encode_at(CUtensorMap* map, const void* base, int nx, int ny, int nz, int box_rows)
{
    StepArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.pre = base;
    return encode_state<ST>(map, a, box_rows);
}

template <int Q, int ST, int V>
cudaError_t launch_t(const StepArgs& a, int zchunk, cudaStream_t s)
{
    using E = typename Storage<ST>::ctype;
    constexpr int H = Shape<Q, E, V>::H;
    constexpr size_t SMEM = tile_smem<Q, ST, H, true>();
    static_assert(SMEM <= 227 * 1024, "shared memory of one block");
    auto kern = tau1_tiled_tma_kernel<Q, ST, H, Shape<Q, E, V>::MINB>;
    // the attribute is per device; setting it on every launch is cheap
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    e = encode_state<ST>(&map, a, 2 * H + 2);
    if (e != cudaSuccess) return e;
    const int ntx = (a.nx + 31) / 32;
    const int ntiles = ntx * ((a.ny + 2 * H - 1) / (2 * H));
    const int chunk = a.nz < zchunk ? a.nz : zchunk;
    const int nchunks = (a.nz + chunk - 1) / chunk;
    const long long blocks = (long long)ntiles * nchunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, 32 * H, SMEM, s>>>(a, ntx, ntiles, chunk, map);
    return cudaGetLastError();
}

template <int Q, int ST>
cudaError_t launch_v(int variant, const StepArgs& a, cudaStream_t s)
{
    if (variant < 0 || variant >= 2 * tile_shapes(ST)) return cudaErrorInvalidValue;
    const int zchunk = variant_chunk(ST, variant);
    if constexpr (ST == ST_F64) {
        return launch_t<Q, ST, 0>(a, zchunk, s);
    } else {
        switch (variant_shape(ST, variant)) {
        case 0: return launch_t<Q, ST, 0>(a, zchunk, s);
        case 1: return launch_t<Q, ST, 1>(a, zchunk, s);
        case 2: return launch_t<Q, ST, 2>(a, zchunk, s);
        case 3: return launch_t<Q, ST, 3>(a, zchunk, s);
        default: return cudaErrorInvalidValue;
        }
    }
}

}  // namespace

bool tau1_tiled_tma_ok(int q, int storage, int variant, const StepArgs& a)
{
    const int th = tile_height(q, storage, variant);
    if (th == 0 || a.nx % 32 != 0 || a.ny % th != 0) return false;
    // a box row of 16-bit records starts at a multiple of 16 bytes only if nx is even
    if ((storage == ST_F16S || storage == ST_BF16S) && a.nx % 2 != 0) return false;
    if ((reinterpret_cast<uintptr_t>(a.pre) & 15) != 0) return false;
    return encode_fn() != nullptr;
}

cudaError_t launch_tau1_tiled_tma(int q, int storage, int variant, const StepArgs& a, cudaStream_t s)
{
    switch (q * 10 + storage) {
    case 190 + ST_F64: return launch_v<19, ST_F64>(variant, a, s);
    case 190 + ST_F32: return launch_v<19, ST_F32>(variant, a, s);
    case 190 + ST_F16S: return launch_v<19, ST_F16S>(variant, a, s);
    case 190 + ST_BF16S: return launch_v<19, ST_BF16S>(variant, a, s);
    case 270 + ST_F64: return launch_v<27, ST_F64>(variant, a, s);
    case 270 + ST_F32: return launch_v<27, ST_F32>(variant, a, s);
    case 270 + ST_F16S: return launch_v<27, ST_F16S>(variant, a, s);
    case 270 + ST_BF16S: return launch_v<27, ST_BF16S>(variant, a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t encode_state_map(int storage, const void* base, int nx, int ny, int nz, int box_rows, CUtensorMap* map)
{
    switch (storage) {
    case ST_F64: return encode_at<ST_F64>(map, base, nx, ny, nz, box_rows);
    case ST_F32: return encode_at<ST_F32>(map, base, nx, ny, nz, box_rows);
    case ST_F16S: return encode_at<ST_F16S>(map, base, nx, ny, nz, box_rows);
    case ST_BF16S: return encode_at<ST_BF16S>(map, base, nx, ny, nz, box_rows);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

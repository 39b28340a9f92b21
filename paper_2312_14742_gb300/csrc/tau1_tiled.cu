// Tiled Tau1 step kernel for one dense box: one block per tile column of the
// tile_column() update (a 32 x 2H tile of the x-y plane, up to 32 planes of z).
//
// Grid: one block per (z-chunk, tile), ordered chunk-major, so the tiles of a
// chunk run side by side and halo reads hit L2.
#include "tile_column.cuh"

namespace lbm {

namespace {

using namespace tile;

template <int Q, int ST, int H, int MINB>
__global__ void __launch_bounds__(32 * H, MINB) tau1_tiled_kernel(StepArgs a, int ntx, int ntiles, int chunk)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int tile = blockIdx.x % ntiles;
    const int z0 = (blockIdx.x / ntiles) * chunk;
    const int z1 = min(a.nz, z0 + chunk);
    const int x0 = (tile % ntx) * 32, y0 = (tile / ntx) * (2 * H);
    const Scales sc(a.dscale);
    float amax[4];
    tile_column<Q, ST, H, false>(a, sc, x0, y0, z0, z1, smem_raw, amax);
}

template <int Q, int ST, int V>
cudaError_t launch_t(const StepArgs& a, int zchunk, cudaStream_t s)
{
    using E = typename Storage<ST>::ctype;
    constexpr int H = Shape<Q, E, V>::H;
    using C = TCfg<Q, 32, H, E>;
    auto kern = tau1_tiled_kernel<Q, ST, H, Shape<Q, E, V>::MINB>;
    // the attribute is per device; setting it on every launch is cheap
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    const int ntx = (a.nx + 31) / 32;
    const int nty = (a.ny + 2 * H - 1) / (2 * H);
    const int ntiles = ntx * nty;
    const int chunk = a.nz < zchunk ? a.nz : zchunk;
    const int nchunks = (a.nz + chunk - 1) / chunk;
    const long long blocks = (long long)ntiles * nchunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, C::NT, C::SMEM, s>>>(a, ntx, ntiles, chunk);
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

bool tau1_tiled_supported(int q, int storage, int64_t n)
{
    return (q == 19 || q == 27) && storage >= ST_F64 && storage <= ST_BF16S && n > 0 && n < ((int64_t)1 << 31);
}

// Variants of a single box: [0, 2R) the row-pair kernel (R tile shapes, then
// 24- or 32-plane chunks), [2R, 2R + 2T) the pair-position kernel (T shapes,
// same chunk rule; staged when the tiles are full). A row-pair variant that
// does not fit the box (ragged tiles) runs the pair-position variant with the
// same chunk height instead.
int tau1_tiled_variants(int, int storage) { return 2 * tau1_rowpair_shapes(storage) + 2 * tile_shapes(storage); }

int tau1_tile_shapes(int storage) { return tile_shapes(storage); }

cudaError_t launch_tau1_tiled(int q, int storage, int variant, const StepArgs& a, cudaStream_t s)
{
    const int nr = tau1_rowpair_shapes(storage);
    if (variant < 0 || variant >= tau1_tiled_variants(q, storage)) return cudaErrorInvalidValue;
    if (variant < 2 * nr) {
        const int shape = variant % nr;
        if (tau1_rowpair_ok(q, storage, shape, a))
            return launch_tau1_rowpair(q, storage, shape, variant < nr ? 24 : 32, a, s);
        variant = variant < nr ? 0 : tile_shapes(storage);
    } else {
        variant -= 2 * nr;
    }
    if (tau1_tiled_tma_ok(q, storage, variant, a)) return launch_tau1_tiled_tma(q, storage, variant, a, s);
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

}  // namespace lbm

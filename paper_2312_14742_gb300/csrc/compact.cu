// Compact porous layout: the dense state records, with the work of a step
// split by tile column (a 32 x H tile of the x-y plane, a chunk of 24 or 32
// z planes: the unit of work of one row-pair kernel variant).
//
// The paper's kernels skip solid chunks and treat mixed chunks through the
// node mask (Section 3.2); its bandwidth model for porous media charges a
// mixed chunk for all of its nodes (Section 4.3, B_est), and its outlook
// (Section 5) names indirect addressing of the fluid nodes. Here each tile
// column is classed by its fluid count c out of m nodes:
//   - c = 0: never visited (no record is read or written);
//   - c >= f* m: stepped by the row-pair kernel through a list of tile
//     columns (every node of the tile is loaded, as in the dense layout);
//   - 0 < c < f* m: its fluid nodes join a node list (4-byte box indices, in
//     z, y, x order of the tile), stepped one thread per node with the
//     neighbours read straight from the dense records (each state copy holds
//     one more record after the box: a solid sentinel for the sources that
//     lie outside a non-periodic face).
// Both kernels compute every link as the dense kernels do, and the node sets
// are disjoint, so a step gives the dense step's bits.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

// n / d for 0 <= n < 2^31 and a divisor d >= 1 fixed per launch, as a
// multiply-high, an add and a shift (Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l; the sum
// stays below 2^32 because n < 2^31.
struct DivBy {
    uint32_t m, l;
    static DivBy make(uint32_t d)
    {
        DivBy r;
        r.l = 0;
        while ((1ull << r.l) < d) ++r.l;
        r.m = (uint32_t)((((1ull << 32) * ((1ull << r.l) - d)) / d) + 1);
        return r;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(m, n) + n) >> l; }
};

// Offsets, relative to a node at coordinate c of an axis of n nodes and
// stride st, of the source coordinate c - v for v = -1, 0, +1 (entry v + 1),
// and whether that source lies in the box (periodic axes wrap).
__device__ __forceinline__ void axis_sources(uint32_t c, uint32_t n, int st, bool per, int off[3], bool in[3])
{
    off[1] = 0;
    in[1] = true;
    // v = +1: source c - 1
    in[2] = c > 0 || per;
    off[2] = c > 0 ? -st : (per ? (int)(n - 1) * st : 0);
    // v = -1: source c + 1
    in[0] = c + 1 < n || per;
    off[0] = c + 1 < n ? st : (per ? -(int)(n - 1) * st : 0);
}

// One Tau1 step of the listed (fluid) box nodes, one thread per node, the
// neighbours' records gathered from the dense state. A source outside a
// non-periodic face is read from the sentinel record n (drho = NaN, u = 0)
// that follows the box in both state copies, so that every source is a plain
// load and a wall is recognised by its NaN alone. A thread issues the loads of
// all q - 1 sources first (FP32 and 16-bit storage; FP64 one link at a time,
// for registers), then evaluates the links in the dense kernels' order
// (c_z = +1, 0, -1, each in k order) with their per-link arithmetic: the
// equilibrium of a fluid source, or the reflected own equilibrium for a wall
// (the dense kernels add these as fma(sigma, b, v) with the other term zero;
// here the term is selected, which gives the same value, the sign of a zero
// term aside).
template <int Q, int ST>
__global__ void __launch_bounds__(256) tau1_list_kernel(StepArgs a, const int* __restrict__ nodes, int count,
                                                        DivBy by_nx, DivBy by_nxy)
{
    using S = Storage<ST>;
    using T = typename S::ctype;
    constexpr bool PRELOAD = sizeof(T) == 4;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const uint32_t i = (uint32_t)__ldg(nodes + t);
    const Scales sc(a.dscale);
    T d0, ux0, uy0, uz0;
    S::load(a.pre, i, sc.inv, d0, ux0, uy0, uz0);
    if (isnan(d0)) return;  // a listed node is fluid; a NaN state is left as it is, as elsewhere
    const uint32_t nx = (uint32_t)a.nx, nxy = nx * (uint32_t)a.ny;
    const uint32_t sentinel = nxy * (uint32_t)a.nz;
    const uint32_t z = by_nxy.div(i), r = i - z * nxy, y = by_nx.div(r), x = r - y * nx;
    int ox[3], oy[3], oz[3];
    bool ix[3], iy[3], iz[3];
    axis_sources(x, nx, 1, a.periodic[0], ox, ix);
    axis_sources(y, (uint32_t)a.ny, (int)nx, a.periodic[1], oy, iy);
    axis_sources(z, (uint32_t)a.nz, (int)nxy, a.periodic[2], oz, iz);

    T rd[Q], rux[Q], ruy[Q], ruz[Q];
    auto gather = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int X = cvel(K, 0) + 1, Y = cvel(K, 1) + 1, Z = cvel(K, 2) + 1;
        const uint32_t s = (ix[X] && iy[Y] && iz[Z]) ? i + (uint32_t)(ox[X] + oy[Y] + oz[Z]) : sentinel;
        S::load(a.pre, s, sc.inv, rd[K], rux[K], ruy[K], ruz[K]);
    };
    if constexpr (PRELOAD) static_for<1, Q>(gather);

    const T gx = gcomp<T>(a, 0), gy = gcomp<T>(a, 1), gz = gcomp<T>(a, 2);
    const NodeMoments<T> own = node_moments<T>(d0, ux0, uy0, uz0, gx, gy, gz);
    NodeAcc<T, Weights<Q>::NCLASS> acc;
    acc.S[0] = own.A;  // rest direction: p = 0

    auto link = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        if constexpr (!PRELOAD) gather(kc);
        const NodeMoments<T> m = node_moments<T>(rd[K], rux[K], ruy[K], ruz[K], gx, gy, gz);
        const T v = feq_scaled(m.A, m.H, dir_dot<K, T>(m.Px, m.Py, m.Pz));
        const T b = feq_scaled(own.A, own.H, -dir_dot<K, T>(own.Px, own.Py, own.Pz));
        acc.template add<Q, K>(isnan(rd[K]) ? b : v);
    };
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 1) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 0) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == -1) link(kc); });

    T d, ux, uy, uz;
    node_finish<Q, T>(acc, d, ux, uy, uz);
    step_store<ST>(a.post, i, d, ux, uy, uz, sc.s, a.seed);
}

// The sentinel record n of a state copy: drho = NaN, u = 0.
template <int ST>
__global__ void sentinel_kernel(void* buf, uint32_t n, const float* __restrict__ dscale)
{
    using T = typename Storage<ST>::ctype;
    const float one[4] = {1.f, 1.f, 1.f, 1.f};
    Storage<ST>::store(buf, n, T(NAN), T(0), T(0), T(0), dscale ? dscale : one);
}

template <int Q, int ST>
cudaError_t launch_list_t(const StepArgs& a, const int* nodes, int count, cudaStream_t s)
{
    const DivBy bx = DivBy::make((uint32_t)a.nx), bxy = DivBy::make((uint32_t)a.nx * (uint32_t)a.ny);
    tau1_list_kernel<Q, ST><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(a, nodes, count, bx, bxy);
    return cudaGetLastError();
}

constexpr int CT = 256;  // threads of the count and list kernels (8 warps)

struct TileGeo {
    int nx, ny, nz, h, chunk, ntx, ntiles;
    __device__ void origin(int b, int& x0, int& y0, int& z0, int& z1) const
    {
        const int tile = b % ntiles;
        z0 = (b / ntiles) * chunk;
        z1 = min(nz, z0 + chunk);
        x0 = (tile % ntx) * 32;
        y0 = (tile / ntx) * h;
    }
    // node of lane x of x-row r of the tile column (rows in z, y order), or -1
    __device__ int64_t node(int x0, int y0, int z0, int r, int lane) const
    {
        const int x = x0 + lane, y = y0 + r % h, z = z0 + r / h;
        if (x >= nx || y >= ny) return -1;
        return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
    }
};

__device__ __forceinline__ bool is_fluid(const uint8_t* flags, int64_t i)
{
    return i >= 0 && !(flags[i] & FLAG_SOLID);
}

// counts[b] = fluid nodes of tile column b; one block per tile column, one
// warp per x-row (coalesced flag bytes).
__global__ void __launch_bounds__(CT) tile_count_kernel(TileGeo g, const uint8_t* __restrict__ flags, int* counts)
{
    __shared__ int part[CT / 32];
    int x0, y0, z0, z1;
    g.origin(blockIdx.x, x0, y0, z0, z1);
    const int rows = g.h * (z1 - z0);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int c = 0;
    for (int r = warp; r < rows; r += CT / 32) c += __popc(__ballot_sync(0xffffffffu, is_fluid(flags, g.node(x0, y0, z0, r, lane))));
    if (lane == 0) part[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < CT / 32; ++w) s += part[w];
        counts[blockIdx.x] = s;
    }
}

// The fluid nodes of the listed tile columns: tile column tiles[j] writes its
// fluid nodes, in row order, to nodes[offsets[j] ...]. One block per tile
// column; a round of 8 rows at a time, one per warp, numbered by a scan of
// the warps' ballot counts.
__global__ void __launch_bounds__(CT) tile_nodes_kernel(TileGeo g, const uint8_t* __restrict__ flags,
                                                        const int* __restrict__ tiles, const int* __restrict__ offsets,
                                                        int* __restrict__ nodes)
{
    __shared__ int part[CT / 32];
    int x0, y0, z0, z1;
    g.origin(tiles[blockIdx.x], x0, y0, z0, z1);
    const int rows = g.h * (z1 - z0);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    int base = offsets[blockIdx.x];
    for (int r0 = 0; r0 < rows; r0 += CT / 32) {
        const int r = r0 + warp;
        const int64_t i = r < rows ? g.node(x0, y0, z0, r, lane) : -1;
        const bool f = is_fluid(flags, i);
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) part[warp] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < CT / 32; ++w) {
            before += w < warp ? part[w] : 0;
            total += part[w];
        }
        if (f) nodes[base + before + __popc(m & ((1u << lane) - 1u))] = (int)i;
        base += total;
        __syncthreads();
    }
}

TileGeo geo_of(const CompactTiles& t, int nx, int ny, int nz)
{
    TileGeo g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.h = t.h;
    g.chunk = nz < t.zchunk ? nz : t.zchunk;
    g.ntx = (nx + 31) / 32;
    g.ntiles = g.ntx * ((ny + g.h - 1) / g.h);
    return g;
}

}  // namespace

CompactTiles compact_tiles(int q, int storage, int variant)
{
    const int nr = tau1_rowpair_shapes(storage);
    CompactTiles t;
    t.shape = variant % nr;
    t.zchunk = variant < nr ? 24 : 32;
    t.h = tau1_rowpair_tile_height(q, storage, t.shape);
    return t;
}

int64_t compact_tile_columns(const CompactTiles& t, int nx, int ny, int nz)
{
    const TileGeo g = geo_of(t, nx, ny, nz);
    if (g.h <= 0) return 0;
    return (int64_t)g.ntiles * ((nz + g.chunk - 1) / g.chunk);
}

int64_t compact_tile_nodes(const CompactTiles& t, int nx, int ny, int nz, int b)
{
    const TileGeo g = geo_of(t, nx, ny, nz);
    const int tile = b % g.ntiles;
    const int z0 = (b / g.ntiles) * g.chunk;
    const int x0 = (tile % g.ntx) * 32, y0 = (tile / g.ntx) * g.h;
    const int64_t w = nx - x0 < 32 ? nx - x0 : 32;
    const int64_t hh = ny - y0 < g.h ? ny - y0 : g.h;
    const int64_t d = nz - z0 < g.chunk ? nz - z0 : g.chunk;
    return w * hh * d;
}

cudaError_t launch_compact_count(const CompactTiles& t, int nx, int ny, int nz, const uint8_t* flags, int* counts,
                                 cudaStream_t s)
{
    const TileGeo g = geo_of(t, nx, ny, nz);
    const int64_t nb = compact_tile_columns(t, nx, ny, nz);
    if (nb <= 0 || nb > 0x7fffffffLL) return cudaErrorInvalidValue;
    tile_count_kernel<<<(unsigned)nb, CT, 0, s>>>(g, flags, counts);
    return cudaGetLastError();
}

cudaError_t launch_compact_nodes(const CompactTiles& t, int nx, int ny, int nz, const uint8_t* flags, const int* tiles,
                                 const int* offsets, int ntiles, int* nodes, cudaStream_t s)
{
    if (ntiles == 0) return cudaSuccess;
    const TileGeo g = geo_of(t, nx, ny, nz);
    tile_nodes_kernel<<<(unsigned)ntiles, CT, 0, s>>>(g, flags, tiles, offsets, nodes);
    return cudaGetLastError();
}

cudaError_t launch_compact_sentinel(int storage, void* buf, int64_t n, const float* dscale, cudaStream_t s)
{
    switch (storage) {
    case ST_F64: sentinel_kernel<ST_F64><<<1, 1, 0, s>>>(buf, (uint32_t)n, dscale); break;
    case ST_F32: sentinel_kernel<ST_F32><<<1, 1, 0, s>>>(buf, (uint32_t)n, dscale); break;
    case ST_F16S: sentinel_kernel<ST_F16S><<<1, 1, 0, s>>>(buf, (uint32_t)n, dscale); break;
    case ST_BF16S: sentinel_kernel<ST_BF16S><<<1, 1, 0, s>>>(buf, (uint32_t)n, dscale); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tau1_list(int q, int storage, const StepArgs& a, const int* nodes, int64_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    // node indices are int32 and nx ny z + y nx + x must not wrap in 32 bits
    if (count > 0x7fffffffLL || (int64_t)a.nx * a.ny * a.nz >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    const int c = (int)count;
    switch (q * 10 + storage) {
    case 190 + ST_F64: return launch_list_t<19, ST_F64>(a, nodes, c, s);
    case 190 + ST_F32: return launch_list_t<19, ST_F32>(a, nodes, c, s);
    case 190 + ST_F16S: return launch_list_t<19, ST_F16S>(a, nodes, c, s);
    case 190 + ST_BF16S: return launch_list_t<19, ST_BF16S>(a, nodes, c, s);
    case 270 + ST_F64: return launch_list_t<27, ST_F64>(a, nodes, c, s);
    case 270 + ST_F32: return launch_list_t<27, ST_F32>(a, nodes, c, s);
    case 270 + ST_F16S: return launch_list_t<27, ST_F16S>(a, nodes, c, s);
    case 270 + ST_BF16S: return launch_list_t<27, ST_BF16S>(a, nodes, c, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

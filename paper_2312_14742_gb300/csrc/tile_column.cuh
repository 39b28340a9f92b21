// Tiled Tau1 step kernel: 2.5D z-march with shared-memory exchange of the
// equilibria each node sends to its in-plane neighbours; every thread updates
// two nodes in the lanes of a two-lane type (packed f32x2 for FP32
// arithmetic, two FP64 lanes for FP64).
//
// Tau1 (Eq. LBMTau1) says the population arriving at x along c_k is
// f_k^eq of the source x - c_k. Each node therefore evaluates its q outgoing
// equilibria once (Eq. feq scaled by 1/w_k, in pairs k / inv(k) that share
// one fma chain) and every destination only gathers and adds. This is the
// buffering of neighbour data inside the processor that the paper's
// complexity analysis (Section 2.1.3) asks for, so that HBM sees one read and
// one write of (rho, u) per node. The velocity is multiplied once by 1/rho
// (Algorithm "Optimized Tau1 ... stores velocity").
//
// Tile = 32 x 2H nodes, block = 32 x H threads; a thread owns the nodes
// (x, y) [lane A] and (x, y + H) [lane B] of the tile and marches in z.
// Shared memory is indexed by "pair positions" (x', y'), x' in [-1, 32],
// y' in [-1, H], lane A = tile node (x', y'), lane B = node (x', y' + H), so
// that both sources x - c_k of a thread sit at one pair position
// (x - c_x, y - c_y). Pair row -1 holds the halo row below (A) and interior
// row H-1 (B); pair row H holds interior row H (A) and the halo row above
// (B). Warp 2 (warp 0 when H < 3) computes both halo rows as one two-lane pair, warp 1 the two
// halo columns; the owners of rows H-1 and H copy their exports into pair
// rows -1 and H. Halo nodes export only the directions pointing into the tile.
//
// At the "arrival" of plane p every position stores, per in-plane direction
// (dx, dy) != 0, its values for c_z = -1, 0, +1 and its solid fraction
// sigma (1 for a solid node or a position beyond a non-periodic face, else
// 0). Solid nodes export 0. After one barrier each thread gathers: c_z = -1
// values complete destination plane p - 1, c_z = 0 values go into plane p,
// c_z = +1 values wait one arrival in registers; (0,0,+-1) and rest never
// leave the thread. Walls (Algorithm "Complete Tau1 ... halfway
// bounce-back") enter every link as fma(sigma, b, v), where v is the
// gathered value and b the destination node's own outgoing value in
// direction inv(k): v for a fluid source, b for a wall, with no branch.
//
#pragma once

#include "kernels.h"
#include "pack2.cuh"
#include "static_for.cuh"
#include "tau1_node.cuh"
#include "tma.cuh"

namespace lbm {

namespace tile {

__host__ __device__ constexpr int kdir(int cx, int cy, int cz)
{
    for (int k = 0; k < 27; ++k)
        if (cvel(k, 0) == cx && cvel(k, 1) == cy && cvel(k, 2) == cz) return k;
    return -1;
}

// Exchange blocks (in-plane direction of block b) and D3Q19 diagonal slots
// (in-plane diagonal j, c_z = 0 only).
template <int Q> struct Xch;
template <> struct Xch<19> {
    static constexpr int NB = 4, ND = 4;
    __host__ __device__ static constexpr int dx(int b) { return b == 0 ? 1 : (b == 1 ? -1 : 0); }
    __host__ __device__ static constexpr int dy(int b) { return b == 2 ? 1 : (b == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int ddx(int j) { return (j == 0 || j == 3) ? 1 : -1; }
    __host__ __device__ static constexpr int ddy(int j) { return (j == 0 || j == 2) ? 1 : -1; }
};
template <> struct Xch<27> {
    static constexpr int NB = 8, ND = 0;
    __host__ __device__ static constexpr int dx(int b)
    {
        return (b == 0 || b == 4 || b == 6) ? 1 : ((b == 1 || b == 5 || b == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int dy(int b)
    {
        return (b == 2 || b == 4 || b == 7) ? 1 : ((b == 3 || b == 5 || b == 6) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ddx(int) { return 0; }
    __host__ __device__ static constexpr int ddy(int) { return 0; }
};
__host__ __device__ constexpr int block_of(int dx, int dy)
{
    return dy == 0 ? (dx > 0 ? 0 : 1) : (dx == 0 ? (dy > 0 ? 2 : 3) : (dx == dy ? (dx > 0 ? 4 : 5) : (dx > 0 ? 6 : 7)));
}
__host__ __device__ constexpr int diag_of(int dx, int dy) { return dx == dy ? (dx > 0 ? 0 : 1) : (dx > 0 ? 3 : 2); }

template <typename E> struct __align__(4 * sizeof(E)) V4 { E x, y, z, w; };
template <typename E> struct __align__(2 * sizeof(E)) V2 { E x, y; };

template <int Q, int TX, int H, typename E> struct TCfg {
    static constexpr int NB = Xch<Q>::NB, ND = Xch<Q>::ND;
    static constexpr int PW = TX + 2;
    static constexpr int NPP = (TX + 2) * (H + 2);  // pair positions
    static constexpr int NT = TX * H;
    // slot: L01[NB][NPP] {c_z=-1: A, B; c_z=0: A, B} | L2[NB][NPP] {c_z=+1: A, B}
    //       | DG[ND][NPP] {A, B} | SG[NPP] {sigma A, sigma B}
    static constexpr size_t L01_BYTES = (size_t)NB * NPP * sizeof(V4<E>);
    static constexpr size_t L2_BYTES = (size_t)NB * NPP * sizeof(V2<E>);
    static constexpr size_t DG_BYTES = (size_t)ND * NPP * sizeof(V2<E>);
    static constexpr size_t SG_BYTES = (size_t)NPP * sizeof(V2<E>);
    static constexpr size_t SLOT_BYTES = L01_BYTES + L2_BYTES + DG_BYTES + SG_BYTES;
    static constexpr size_t SMEM = 2 * SLOT_BYTES;
    static_assert(TX == 32, "a warp is one tile row");
    static_assert(H >= 2 && 2 * (H + 2) <= 32, "warp 1 holds both halo columns");
};

// Staged (TMA) mode: each plane's box of raw records, x0 - XOFF .. x0 + 31 +
// XOFF by y0 - 1 .. y0 + 2H, copied by the tensor unit into one of NSTAGE
// buffers two planes ahead of its use. A box row starts at element 4 (x0 -
// XOFF); the copy needs that to be a multiple of 16 bytes: XOFF = 1 for
// records of 16 or 32 bytes, 2 for the 8-byte records of 16-bit storage
// (x0 is a multiple of 32).
template <int ST, int H> struct StageCfg {
    static constexpr int REC = Storage<ST>::NODE_BYTES;  // one record: 4 values
    static constexpr int XOFF = REC >= 16 ? 1 : 2;
    static constexpr int SW = 32 + 2 * XOFF, SROWS = 2 * H + 2, NSTAGE = 3;
    static constexpr int BOX_X = 4 * SW;                  // box width in elements
    static constexpr uint32_t BOX_BYTES = (uint32_t)(SW * SROWS * REC);
    static constexpr size_t STAGE_BYTES = (BOX_BYTES + 127) / 128 * 128;
    static_assert((4 * XOFF * (REC / 4)) % 16 == 0 && (SW * REC) % 16 == 0, "box alignment");
};

// Dynamic shared memory of tile_column: exchange slots, then (TMA) up to 128
// bytes of alignment padding, the stages and their mbarriers.
template <int Q, int ST, int H, bool TMA> __host__ __device__ constexpr size_t tile_smem()
{
    using C = TCfg<Q, 32, H, typename Storage<ST>::ctype>;
    using SC = StageCfg<ST, H>;
    return TMA ? C::SMEM + 128 + SC::NSTAGE * SC::STAGE_BYTES + 8 * SC::NSTAGE : C::SMEM;
}

// Stage buffers and their mbarriers inside tile_column's shared memory.
template <int Q, int ST, int H> __device__ __forceinline__ unsigned char* stage_base(unsigned char* smem_raw)
{
    using C = TCfg<Q, 32, H, typename Storage<ST>::ctype>;
    const uint32_t sbase = smem_u32(smem_raw);
    return smem_raw + (((sbase + (uint32_t)C::SMEM + 127u) & ~127u) - sbase);
}
template <int Q, int ST, int H> __device__ __forceinline__ uint64_t* stage_barriers(unsigned char* smem_raw)
{
    using SC = StageCfg<ST, H>;
    return reinterpret_cast<uint64_t*>(stage_base<Q, ST, H>(smem_raw) + SC::NSTAGE * SC::STAGE_BYTES);
}
// Initialises the stage mbarriers (thread 0; the caller synchronises the block
// before the first tile_column). Their phases then run on across calls: each
// call takes and returns the phase bits.
template <int Q, int ST, int H> __device__ __forceinline__ void stage_init(unsigned char* smem_raw)
{
    if (threadIdx.x == 0) {
        uint64_t* mbar = stage_barriers<Q, ST, H>(smem_raw);
#pragma unroll
        for (int st = 0; st < StageCfg<ST, H>::NSTAGE; ++st) mbar_init(&mbar[st], 1);
        mbar_init_fence();
    }
}

__device__ __forceinline__ int ppos(int tx, int ty, int pw) { return (ty + 1) * pw + (tx + 1); }

__device__ __forceinline__ bool wrap_coord(int& c, int n, int periodic)
{
    if (c >= 0 && c < n) return true;
    if (!periodic) return false;
    c %= n;
    if (c < 0) c += n;
    return true;
}

// Raw state of the two nodes (lanes A, B) of one thread or halo slot.
template <typename L> struct Raw2 {
    L d, ux, uy, uz;
};

template <int ST, typename E>
__device__ __forceinline__ void load_node(const StepArgs& a, const Scales& sc, bool ok, uint32_t i, E& d, E& ux, E& uy,
                                          E& uz)
{
    if (ok) {
        Storage<ST>::load(a.pre, i, sc.inv, d, ux, uy, uz);
    } else {
        d = E(NAN);  // beyond a non-periodic face: a wall, like a solid node
        ux = uy = uz = E(0);
    }
}

// Two-lane moments of a raw pair; solid lanes (drho NaN) get A = P = 0, so
// all their outgoing values are exactly 0, and sigma = 1.
template <typename L>
__device__ __forceinline__ NodeMoments<L> moments_of(Raw2<L> r, const L& g0, const L& g1, const L& g2, L& sigma)
{
    using E = typename L::elem;
    const bool sA = isnan(r.d.v.x), sB = isnan(r.d.v.y);
    r.d = L(sA ? E(0) : r.d.v.x, sB ? E(0) : r.d.v.y);
    const L keep(sA ? E(0) : E(1), sB ? E(0) : E(1));
    sigma = L(sA ? E(1) : E(0), sB ? E(1) : E(0));
    NodeMoments<L> m = node_moments<L>(r.d, r.ux, r.uy, r.uz, g0, g1, g2);
    m.A = m.A * keep;
    m.Px = m.Px * keep;
    m.Py = m.Py * keep;
    m.Pz = m.Pz * keep;
    return m;
}

template <typename E>
__device__ __forceinline__ void track_amax(float (&m)[4], E d, E ux, E uy, E uz)
{
    m[0] = fmaxf(m[0], fabsf((float)d));
    m[1] = fmaxf(m[1], fabsf((float)ux));
    m[2] = fmaxf(m[2], fabsf((float)uy));
    m[3] = fmaxf(m[3], fabsf((float)uz));
}

// One tile column of one step: the tile (x0, y0) of the box, planes
// z0 <= z < z1. All threads of the block call it together (it synchronises);
// smem_raw holds tile_smem<Q, ST, H, TMA>() bytes, 128-byte aligned. With
// AMAX, amax[f] collects the largest |value| of field f among the nodes this
// thread stores. With TMA the raw records come from shared-memory stages
// (initialised by stage_init; *phase_io carries their phase bits from call
// to call) filled by the tensor unit through tmap (the state read, viewed as a
// 3D array of 4 nx x ny x nz values); the tile must lie inside the box, and
// halo nodes outside it are read from global memory (periodic images) or are
// walls. A wait that runs out is counted in *a.timeouts, and the thread then
// tries no later wait and stores nothing more in this call.
template <int Q, int ST, int H, bool AMAX, bool TMA = false>
__device__ __forceinline__ void tile_column(const StepArgs& a, const Scales& sc, int x0, int y0, int z0, int z1,
                                            unsigned char* smem_raw, float (&amax)[4],
                                            const CUtensorMap* tmap = nullptr, uint32_t* phase_io = nullptr)
{
    constexpr int TX = 32;
    using S = Storage<ST>;
    using E = typename S::ctype;
    using L = typename Lanes<E>::type;
    using C = TCfg<Q, TX, H, E>;
    using X = Xch<Q>;
    constexpr int NPP = C::NPP, PW = C::PW, NB = C::NB, ND = C::ND;
    constexpr int NC = Weights<Q>::NCLASS;
    constexpr int KZP = kdir(0, 0, 1), KZM = kdir(0, 0, -1);
    constexpr int TY = 2 * H;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;  // pair row = warp index
    const int my = ppos(tx, ty, PW);

    const uint32_t nxy = (uint32_t)a.nx * (uint32_t)a.ny;
    const int gx = x0 + tx, gyA = y0 + ty, gyB = y0 + ty + H;
    const bool activeA = gx < a.nx && gyA < a.ny;
    const bool activeB = gx < a.nx && gyB < a.ny;
    const L g0(gcomp<E>(a, 0)), g1(gcomp<E>(a, 1)), g2(gcomp<E>(a, 2));

    // in-plane offsets, wrapped once
    auto xy_of = [&](int x, int y, bool& ok) -> uint32_t {
        ok = wrap_coord(x, a.nx, a.periodic[0]) && wrap_coord(y, a.ny, a.periodic[1]);
        return (uint32_t)x + (uint32_t)a.nx * (uint32_t)y;
    };
    bool okA, okB;
    const uint32_t xyA = xy_of(gx, gyA, okA), xyB = xy_of(gx, gyB, okB);

    // halo roles. Warp 2 (warp 0 if H < 3): halo rows below (lane A) and above (lane B).
    // Warp 1: halo columns, lanes 0..H+1 left (x = -1), H+2..2H+3 right (x = 32).
    const bool hrow = ty == (H >= 3 ? 2 : 0);  // not warp 0, which also stores a duplicated row
    const bool hcol = ty == 1 && tx < 2 * (H + 2);
    const int hcs = tx < H + 2 ? 1 : -1;  // column ring exports directions with dx = hcs
    const int hctx = tx < H + 2 ? -1 : TX;
    const int hcty = tx < H + 2 ? tx - 1 : tx - (H + 2) - 1;
    bool hokA = false, hokB = false;
    uint32_t hxyA = 0, hxyB = 0;
    if (hrow) {
        hxyA = xy_of(gx, y0 - 1, hokA);
        hxyB = xy_of(gx, y0 + TY, hokB);
    } else if (hcol) {
        hxyA = xy_of(x0 + hctx, y0 + hcty, hokA);
        hxyB = xy_of(x0 + hctx, y0 + hcty + H, hokB);
    }
    const bool has_halo = hrow || hcol;
    const int hc_pos = ppos(hctx, hcty, PW);
    const int hc_b0 = hcs > 0 ? block_of(1, 0) : block_of(-1, 0);
    const int hc_bp = (Q == 27) ? (hcs > 0 ? block_of(1, 1) : block_of(-1, 1)) : (hcs > 0 ? diag_of(1, 1) : diag_of(-1, 1));
    const int hc_bm = (Q == 27) ? (hcs > 0 ? block_of(1, -1) : block_of(-1, -1))
                                : (hcs > 0 ? diag_of(1, -1) : diag_of(-1, -1));

    Raw2<L> r_own, r_halo;
    auto prefetch = [&](int p) {
        int gz = p;
        const bool zok = wrap_coord(gz, a.nz, a.periodic[2]);
        const uint32_t zoff = (uint32_t)gz * nxy;
        load_node<ST>(a, sc, zok && okA, zoff + xyA, r_own.d.v.x, r_own.ux.v.x, r_own.uy.v.x, r_own.uz.v.x);
        load_node<ST>(a, sc, zok && okB, zoff + xyB, r_own.d.v.y, r_own.ux.v.y, r_own.uy.v.y, r_own.uz.v.y);
        if (has_halo) {
            load_node<ST>(a, sc, zok && hokA, zoff + hxyA, r_halo.d.v.x, r_halo.ux.v.x, r_halo.uy.v.x, r_halo.uz.v.x);
            load_node<ST>(a, sc, zok && hokB, zoff + hxyB, r_halo.d.v.y, r_halo.ux.v.y, r_halo.uy.v.y, r_halo.uz.v.y);
        }
    };

    // ---- staged (TMA) mode ---------------------------------------------------------
    using SC = StageCfg<ST, H>;
    [[maybe_unused]] unsigned char* stages = nullptr;
    [[maybe_unused]] uint64_t* mbar = nullptr;
    [[maybe_unused]] uint32_t phase = 0;   // bit s: parity of stage s's next completion
    [[maybe_unused]] bool timed_out = false;
    // stage cell (column c, row r) of a halo node; in_box: unwrapped position inside the box
    [[maybe_unused]] int hcA = 0, hrA = 0, hcB = 0, hrB = 0;
    [[maybe_unused]] bool hinA = false, hinB = false;
    if constexpr (TMA) {
        stages = stage_base<Q, ST, H>(smem_raw);
        mbar = stage_barriers<Q, ST, H>(smem_raw);
        phase = *phase_io;
        auto inside = [&](int x, int y) { return x >= 0 && x < a.nx && y >= 0 && y < a.ny; };
        if (hrow) {
            hcA = tx + SC::XOFF; hrA = 0; hinA = inside(gx, y0 - 1);
            hcB = tx + SC::XOFF; hrB = TY + 1; hinB = inside(gx, y0 + TY);
        } else if (hcol) {
            hcA = hctx + SC::XOFF; hrA = hcty + 1; hinA = inside(x0 + hctx, y0 + hcty);
            hcB = hctx + SC::XOFF; hrB = hcty + H + 1; hinB = inside(x0 + hctx, y0 + hcty + H);
        }
    }
    // thread 0 starts the copy of plane p's box into its stage
    [[maybe_unused]] auto issue = [&](int p) {
        int gz = p;
        if (tid == 0 && !timed_out && wrap_coord(gz, a.nz, a.periodic[2])) {
            const int st = (p - z0 + 1) % SC::NSTAGE;
            mbar_arrive_expect_tx(&mbar[st], SC::BOX_BYTES);
            tma_load_3d(stages + st * SC::STAGE_BYTES, tmap, &mbar[st], 4 * (x0 - SC::XOFF), y0 - 1, gz);
        }
    };
    // waits for plane p's box and reads this thread's own and halo records; halo
    // nodes outside the box (across a periodic face) are read from global memory
    [[maybe_unused]] auto fetch_staged = [&](int p) {
        int gz = p;
        const bool zok = wrap_coord(gz, a.nz, a.periodic[2]);
        const uint32_t zoff = (uint32_t)gz * nxy;
        if (!zok) {
            load_node<ST>(a, sc, false, 0, r_own.d.v.x, r_own.ux.v.x, r_own.uy.v.x, r_own.uz.v.x);
            load_node<ST>(a, sc, false, 0, r_own.d.v.y, r_own.ux.v.y, r_own.uy.v.y, r_own.uz.v.y);
            load_node<ST>(a, sc, false, 0, r_halo.d.v.x, r_halo.ux.v.x, r_halo.uy.v.x, r_halo.uz.v.x);
            load_node<ST>(a, sc, false, 0, r_halo.d.v.y, r_halo.ux.v.y, r_halo.uy.v.y, r_halo.uz.v.y);
            return;
        }
        const int st = (p - z0 + 1) % SC::NSTAGE;
        // after a wait ran out, no later wait is tried and nothing more is stored
        if (!timed_out) {
            if (!mbar_wait_bounded(&mbar[st], (phase >> st) & 1u)) timed_out = true;
            phase ^= 1u << st;
        }
        const unsigned char* base = stages + st * SC::STAGE_BYTES;
        auto cell = [&](int c, int r) { return base + (size_t)(r * SC::SW + c) * SC::REC; };
        S::load_at(cell(tx + SC::XOFF, ty + 1), sc.inv, r_own.d.v.x, r_own.ux.v.x, r_own.uy.v.x, r_own.uz.v.x);
        S::load_at(cell(tx + SC::XOFF, ty + H + 1), sc.inv, r_own.d.v.y, r_own.ux.v.y, r_own.uy.v.y, r_own.uz.v.y);
        if (has_halo) {
            if (hinA) S::load_at(cell(hcA, hrA), sc.inv, r_halo.d.v.x, r_halo.ux.v.x, r_halo.uy.v.x, r_halo.uz.v.x);
            else load_node<ST>(a, sc, hokA, zoff + hxyA, r_halo.d.v.x, r_halo.ux.v.x, r_halo.uy.v.x, r_halo.uz.v.x);
            if (hinB) S::load_at(cell(hcB, hrB), sc.inv, r_halo.d.v.y, r_halo.ux.v.y, r_halo.uy.v.y, r_halo.uz.v.y);
            else load_node<ST>(a, sc, hokB, zoff + hxyB, r_halo.d.v.y, r_halo.ux.v.y, r_halo.uy.v.y, r_halo.uz.v.y);
        }
    };

    if constexpr (TMA) {
        issue(z0 - 1);
        issue(z0);
    } else {
        prefetch(z0 - 1);
    }

    NodeAcc<L, NC> acc;  // plane p - 1, all but its c_z = -1 links
    L up_v[Q], up_s[Q];  // c_z = +1 links gathered for plane p: value, source sigma
    L own_in[Q];         // own outgoing (., ., +1) of plane p - 1
    L sig;               // own sigma of plane p (1 = solid or outside)
    L out[Q];            // own outgoing values of plane p
    bool fluidA = false, fluidB = false, fluidA_prev = false, fluidB_prev = false;
#pragma unroll
    for (int k = 0; k < Q; ++k) up_v[k] = up_s[k] = own_in[k] = L(E(0));
    acc.clear();

    struct Slot {
        V4<E>* L01;
        V2<E>* L2;
        V2<E>* DG;
        V2<E>* SG;
    };
    auto slot_of = [&](int p) {
        unsigned char* base = smem_raw + (size_t)((p - z0 + 1) & 1) * C::SLOT_BYTES;
        return Slot{reinterpret_cast<V4<E>*>(base), reinterpret_cast<V2<E>*>(base + C::L01_BYTES),
                    reinterpret_cast<V2<E>*>(base + C::L01_BYTES + C::L2_BYTES),
                    reinterpret_cast<V2<E>*>(base + C::L01_BYTES + C::L2_BYTES + C::DG_BYTES)};
    };

    // Arrival of plane p: own moments and outgoing values, exports to the slot
    // of plane p (own, duplicated pair rows, halo), then the next plane's loads.
    auto export_plane = [&](int p, bool next) {
        if constexpr (TMA) fetch_staged(p);
        const Slot sl = slot_of(p);
        V4<E>* L01 = sl.L01;
        V2<E>* L2 = sl.L2;
        V2<E>* DG = sl.DG;
        V2<E>* SG = sl.SG;
            // ---- own outgoing values (registers) and exports --------------------
            {
                const NodeMoments<L> m = moments_of(r_own, g0, g1, g2, sig);
                out[0] = m.A;
                static_for<0, (Q - 1) / 2>([&](auto ic) {
                    constexpr int K = 1 + 2 * decltype(ic)::value;  // K + 1 = inv(K)
                    const L pk = dir_dot<K, L>(m.Px, m.Py, m.Pz);
                    const L e = fma(pk * m.H, pk, m.A);
                    out[K] = e + pk;
                    out[K + 1] = e - pk;
                });
            }
            fluidA = activeA && sig.v.x == E(0);
            fluidB = activeB && sig.v.y == E(0);
            static_for<0, NB>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                constexpr int dx = X::dx(b), dy = X::dy(b);
                const L vm = out[kdir(dx, dy, -1)], v0 = out[kdir(dx, dy, 0)], vp = out[kdir(dx, dy, 1)];
                L01[b * NPP + my] = V4<E>{vm.v.x, vm.v.y, v0.v.x, v0.v.y};
                L2[b * NPP + my] = V2<E>{vp.v.x, vp.v.y};
            });
            static_for<0, ND>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                const L v = out[kdir(X::ddx(j), X::ddy(j), 0)];
                DG[j * NPP + my] = V2<E>{v.v.x, v.v.y};
            });
            SG[my] = V2<E>{sig.v.x, sig.v.y};
            // interior rows H-1 and H also appear in pair rows -1 (lane B) and H (lane A)
            if (ty == H - 1) {
                const int q = ppos(tx, -1, PW);
                static_for<0, NB>([&](auto bc) {
                    constexpr int b = decltype(bc)::value;
                    if constexpr (X::dy(b) == 1) {
                        L01[b * NPP + q].y = out[kdir(X::dx(b), 1, -1)].v.x;
                        L01[b * NPP + q].w = out[kdir(X::dx(b), 1, 0)].v.x;
                        L2[b * NPP + q].y = out[kdir(X::dx(b), 1, 1)].v.x;
                    }
                });
                static_for<0, ND>([&](auto jc) {
                    constexpr int j = decltype(jc)::value;
                    if constexpr (X::ddy(j) == 1) DG[j * NPP + q].y = out[kdir(X::ddx(j), 1, 0)].v.x;
                });
                SG[q].y = sig.v.x;
            }
            if (ty == 0) {
                const int q = ppos(tx, H, PW);
                static_for<0, NB>([&](auto bc) {
                    constexpr int b = decltype(bc)::value;
                    if constexpr (X::dy(b) == -1) {
                        L01[b * NPP + q].x = out[kdir(X::dx(b), -1, -1)].v.y;
                        L01[b * NPP + q].z = out[kdir(X::dx(b), -1, 0)].v.y;
                        L2[b * NPP + q].x = out[kdir(X::dx(b), -1, 1)].v.y;
                    }
                });
                static_for<0, ND>([&](auto jc) {
                    constexpr int j = decltype(jc)::value;
                    if constexpr (X::ddy(j) == -1) DG[j * NPP + q].x = out[kdir(X::ddx(j), -1, 0)].v.y;
                });
                SG[q].x = sig.v.y;
            }

            // ---- halo exports ----------------------------------------------------
            if (hrow) {
                // lane A: the row below, directions with dy = +1; lane B: the row above, dy = -1
                L hs;
                const NodeMoments<L> m = moments_of(r_halo, g0, g1, g2, hs);
                const L pa = m.Py * L(E(1), E(-1));
                const L pb = m.Px;
                auto f = [&](L pv) { return feq_scaled(m.A, m.H, pv); };
                const int qA = ppos(tx, -1, PW), qB = ppos(tx, H, PW);
                auto put = [&](int bA, int bB, L vm, L v0, L vp) {
                    L01[bA * NPP + qA].x = vm.v.x;
                    L01[bA * NPP + qA].z = v0.v.x;
                    L2[bA * NPP + qA].x = vp.v.x;
                    L01[bB * NPP + qB].y = vm.v.y;
                    L01[bB * NPP + qB].w = v0.v.y;
                    L2[bB * NPP + qB].y = vp.v.y;
                };
                put(block_of(0, 1), block_of(0, -1), f(pa - m.Pz), f(pa), f(pa + m.Pz));
                const L pp = pa + pb, pm = pa - pb;
                if constexpr (Q == 27) {
                    put(block_of(1, 1), block_of(1, -1), f(pp - m.Pz), f(pp), f(pp + m.Pz));
                    put(block_of(-1, 1), block_of(-1, -1), f(pm - m.Pz), f(pm), f(pm + m.Pz));
                } else {
                    const L vpp = f(pp), vpm = f(pm);
                    DG[diag_of(1, 1) * NPP + qA].x = vpp.v.x;
                    DG[diag_of(1, -1) * NPP + qB].y = vpp.v.y;
                    DG[diag_of(-1, 1) * NPP + qA].x = vpm.v.x;
                    DG[diag_of(-1, -1) * NPP + qB].y = vpm.v.y;
                }
                SG[qA].x = hs.v.x;
                SG[qB].y = hs.v.y;
            } else if (hcol) {
                // both lanes: directions with dx = hcs
                L hs;
                const NodeMoments<L> m = moments_of(r_halo, g0, g1, g2, hs);
                const L pa = m.Px * L(E(hcs));
                const L pb = m.Py;
                auto f = [&](L pv) { return feq_scaled(m.A, m.H, pv); };
                auto put = [&](int b, L vm, L v0, L vp) {
                    L01[b * NPP + hc_pos] = V4<E>{vm.v.x, vm.v.y, v0.v.x, v0.v.y};
                    L2[b * NPP + hc_pos] = V2<E>{vp.v.x, vp.v.y};
                };
                put(hc_b0, f(pa - m.Pz), f(pa), f(pa + m.Pz));
                const L pp = pa + pb, pm = pa - pb;
                if constexpr (Q == 27) {
                    put(hc_bp, f(pp - m.Pz), f(pp), f(pp + m.Pz));
                    put(hc_bm, f(pm - m.Pz), f(pm), f(pm + m.Pz));
                } else {
                    const L vpp = f(pp), vpm = f(pm);
                    DG[hc_bp * NPP + hc_pos] = V2<E>{vpp.v.x, vpp.v.y};
                    DG[hc_bm * NPP + hc_pos] = V2<E>{vpm.v.x, vpm.v.y};
                }
                SG[hc_pos] = V2<E>{hs.v.x, hs.v.y};
            }
        if constexpr (TMA) {
            if (p + 2 <= z1) issue(p + 2);
        } else {
            if (next) prefetch(p + 1);
        }
    };

    // The c_z = +1 values of plane p (read after its barrier) wait in registers
    // for plane p + 1; so do the own outgoing (., ., +1) values for its bounce-back.
    auto carry = [&](const Slot& sl, const V2<E> (&fsg)[NB]) {
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int dx = X::dx(b), dy = X::dy(b), K = kdir(dx, dy, 1);
            const V2<E> v = sl.L2[b * NPP + ppos(tx - dx, ty - dy, PW)];
            up_v[K] = L(v.x, v.y);
            up_s[K] = L(fsg[b].x, fsg[b].y);
        });
        up_v[KZP] = out[KZP];
        up_s[KZP] = sig;
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 1) own_in[K] = out[K];
        });
    };

    // Each in-plane source position of this thread, read once per plane:
    // {c_z = -1, c_z = 0} values and sigma.
    auto load_faces = [&](const Slot& sl, V4<E> (&f01)[NB], V2<E> (&fsg)[NB]) {
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            const int q = ppos(tx - X::dx(b), ty - X::dy(b), PW);
            f01[b] = sl.L01[b * NPP + q];
            fsg[b] = sl.SG[q];
        });
    };

    // c_z = -1 values of plane p complete plane p - 1, which is stored if it is
    // this block's and fluid.
    auto finish_prev = [&](int p, const V4<E> (&f01)[NB], const V2<E> (&fsg)[NB]) {
        L dn_v[Q], dn_s[Q];
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int K = kdir(X::dx(b), X::dy(b), -1);
            dn_v[K] = L(f01[b].x, f01[b].y);
            dn_s[K] = L(fsg[b].x, fsg[b].y);
        });
        dn_v[KZM] = out[KZM];  // (0,0,-1): from the own node at plane p
        dn_s[KZM] = sig;
        // bounce values: own outgoing of plane p - 1 in direction inv(k) = (., ., +1)
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == -1) acc.template add<Q, K>(fma(dn_s[K], own_in[inv_dir(K)], dn_v[K]));
        });
        L d_, x_, y_, z_;
        node_finish<Q, L>(acc, d_, x_, y_, z_);
        const uint32_t zoff = (uint32_t)(p - 1) * nxy;
        if (fluidA_prev && !timed_out) {
            step_store<ST>(a.post, zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyA, d_.v.x, x_.v.x, y_.v.x,
                           z_.v.x, sc.s, a.seed);
            if constexpr (AMAX) track_amax(amax, d_.v.x, x_.v.x, y_.v.x, z_.v.x);
        }
        if (fluidB_prev && !timed_out) {
            step_store<ST>(a.post, zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyB, d_.v.y, x_.v.y, y_.v.y,
                           z_.v.y, sc.s, a.seed);
            if constexpr (AMAX) track_amax(amax, d_.v.y, x_.v.y, y_.v.y, z_.v.y);
        }
    };

    // plane p: the c_z = +1 links gathered last arrival, then c_z = 0
    auto start_plane = [&](const Slot& sl, const V4<E> (&f01)[NB], const V2<E> (&fsg)[NB]) {
        acc.S[0] = out[0];
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 1) acc.template add<Q, K>(fma(up_s[K], out[inv_dir(K)], up_v[K]));
        });
        L mid_v[Q], mid_s[Q];
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int K = kdir(X::dx(b), X::dy(b), 0);
            mid_v[K] = L(f01[b].z, f01[b].w);
            mid_s[K] = L(fsg[b].x, fsg[b].y);
        });
        static_for<0, ND>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            constexpr int dx = X::ddx(j), dy = X::ddy(j), K = kdir(dx, dy, 0);
            const int q = ppos(tx - dx, ty - dy, PW);
            const V2<E> v = sl.DG[j * NPP + q];
            const V2<E> s = sl.SG[q];
            mid_v[K] = L(v.x, v.y);
            mid_s[K] = L(s.x, s.y);
        });
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 0) acc.template add<Q, K>(fma(mid_s[K], out[inv_dir(K)], mid_v[K]));
        });
    };

    // plane z0 - 1 (below the chunk): exports and carry only
    export_plane(z0 - 1, true);
    __syncthreads();
    {
        const Slot sl = slot_of(z0 - 1);
        V4<E> f01[NB];
        V2<E> fsg[NB];
        load_faces(sl, f01, fsg);
        carry(sl, fsg);
    }
    // planes of the chunk; the first finish_prev completes plane z0 - 1,
    // which is not this block's (fluid*_prev are false) and is not stored
    for (int p = z0; p < z1; ++p) {
        export_plane(p, true);
        __syncthreads();
        const Slot sl = slot_of(p);
        V4<E> f01[NB];
        V2<E> fsg[NB];
        load_faces(sl, f01, fsg);
        finish_prev(p, f01, fsg);
        start_plane(sl, f01, fsg);
        carry(sl, fsg);
        fluidA_prev = fluidA;
        fluidB_prev = fluidB;
    }
    // plane z1 (above the chunk): its c_z = -1 values finish plane z1 - 1
    export_plane(z1, false);
    __syncthreads();
    {
        const Slot sl = slot_of(z1);
        V4<E> f01[NB];
        V2<E> fsg[NB];
        load_faces(sl, f01, fsg);
        finish_prev(z1, f01, fsg);
    }
    if constexpr (TMA) {
        if (timed_out && a.timeouts) atomicAdd(a.timeouts, 1u);
        *phase_io = phase;
    }
}

// Tile-shape variants (H = half tile height, MINB = resident blocks the
// register budget is sized for). The autotuner picks one per handle
// (single box) or per batch.
template <int Q, typename E, int V> struct Shape;
template <> struct Shape<19, float, 0> { static constexpr int H = 4, MINB = 3; };
template <> struct Shape<19, float, 1> { static constexpr int H = 8, MINB = 1; };
template <> struct Shape<19, float, 2> { static constexpr int H = 8, MINB = 2; };
template <> struct Shape<19, float, 3> { static constexpr int H = 6, MINB = 2; };
template <> struct Shape<27, float, 0> { static constexpr int H = 4, MINB = 2; };
template <> struct Shape<27, float, 1> { static constexpr int H = 8, MINB = 1; };
template <> struct Shape<27, float, 2> { static constexpr int H = 2, MINB = 4; };
template <> struct Shape<27, float, 3> { static constexpr int H = 4, MINB = 3; };
template <int V> struct Shape<19, double, V> { static constexpr int H = 4, MINB = 1; };
template <int V> struct Shape<27, double, V> { static constexpr int H = 2, MINB = 1; };
constexpr int SHAPE_VARIANTS = 4;  // FP32-arithmetic formats; FP64 has one

// Variants of the single-box kernels: a tile shape and the z-chunk height of
// a block (planes per tile column). Variants [0, shapes) use 24-plane chunks,
// [shapes, 2 shapes) 32-plane chunks: more, shorter blocks fill the last wave
// of the grid better, at 2 halo planes per chunk (24 was 2% faster than 32 on
// a 256^3 box). The batched kernel chooses its chunk itself.
inline int tile_shapes(int storage) { return storage == ST_F64 ? 1 : SHAPE_VARIANTS; }
inline int variant_shape(int storage, int variant) { return variant % tile_shapes(storage); }
inline int variant_chunk(int storage, int variant) { return variant < tile_shapes(storage) ? 24 : 32; }

// Tile height 2H of a variant (0 if there is no such variant).
inline int tile_height(int q, int storage, int variant)
{
    if (variant < 0 || variant >= 2 * tile_shapes(storage)) return 0;
    variant = variant_shape(storage, variant);
    if (storage == ST_F64) return variant == 0 ? 2 * (q == 19 ? Shape<19, double, 0>::H : Shape<27, double, 0>::H) : 0;
    if (variant >= SHAPE_VARIANTS) return 0;
    constexpr int h19[4] = {Shape<19, float, 0>::H, Shape<19, float, 1>::H, Shape<19, float, 2>::H,
                            Shape<19, float, 3>::H};
    constexpr int h27[4] = {Shape<27, float, 0>::H, Shape<27, float, 1>::H, Shape<27, float, 2>::H,
                            Shape<27, float, 3>::H};
    return 2 * (q == 19 ? h19[variant] : h27[variant]);
}

}  // namespace tile

}  // namespace lbm

// Row-pair Tau1 step kernel: 2.5D z-march in which each thread owns two
// adjacent rows of one column (lanes A = (x, y), B = (x, y + 1) of a
// two-lane type: packed f32x2 for FP32 arithmetic, two FP64 lanes for FP64)
// and the values each node sends to its neighbours move by warp shuffles
// within a row and through shared memory only across the seams between warps.
//
// Tau1 (Eq. LBMTau1): the population arriving at x along c_k is f_k^eq of
// the source x - c_k. Each node evaluates its q outgoing equilibria once
// (Eq. feq scaled by 1/w_k, in pairs k / inv(k) that share one fma chain)
// and every destination only gathers and adds, so HBM sees one read and one
// write of (rho, u) per node (the buffering that the complexity analysis of
// Section 2.1.3 assumes). Where a value comes from:
//
//   - c_z = 0 rows of the tile: from lane x - c_x of the same warp (shuffle);
//     between rows A and B of one thread: registers;
//   - between the B row of warp w - 1 and the A row of warp w (seam w): the
//     sender stores its values for c_y = +1 (or -1) in shared memory, the
//     receiver loads them after the plane barrier;
//   - c_z = +-1: the z-march keeps them in registers for one plane;
//   - lanes 0 and 31 take the values of the columns x0 - 1 and x0 + 32 from
//     shared memory, where a halo task put them.
//
// Halo tasks (per plane): warp W - 1 computes the rows y0 - 1 and y0 + 2W
// as one two-lane pair and stores their exports into seams 0 and W; warp
// W - 2 computes the columns x0 - 1 and x0 + 32 and the four corners. Halo
// nodes export only the directions pointing into the tile. A halo value is
// computed with the same operations as the owner's value, so every link gets
// the same bits as in the other kernels of this library.
//
// Walls (Algorithm "Complete Tau1 ... halfway bounce-back") enter every link
// as fma(sigma, b, v): v the gathered value (0 from a solid source), b the
// destination's own outgoing value in direction inv(k), sigma = 1 for a solid
// source or one beyond a non-periodic face. Each node is accumulated in the
// order of acc_order() and finished by node_finish(), as in the other step
// kernels (Algorithm "Optimized Tau1 ... stores velocity": one reciprocal).
//
// The raw records of each plane come into shared memory by TMA
// (cp.async.bulk.tensor.3d), a box of the tile plus its one-node halo ring,
// two planes ahead of their use. The tile must lie inside the box
// (nx a multiple of 32, ny of 2W).
#pragma once

#include "tile_column.cuh"

namespace lbm {

namespace rp {

using tile::kdir;

// Number of c_z values carried by in-plane direction (dx, dy) != 0, and the
// index of c_z among them.
template <int Q> __host__ __device__ constexpr int nzv(int dx, int dy)
{
    return (Q == 27 || dx == 0 || dy == 0) ? 3 : 1;
}
template <int Q> __host__ __device__ constexpr int czi(int dx, int dy, int cz)
{
    return nzv<Q>(dx, dy) == 3 ? cz + 1 : 0;
}
// slot of the x component in a seam side: 0 (c_x = 0), 1 (+1), 2 (-1)
__host__ __device__ constexpr int jx(int dx) { return dx == 0 ? 0 : (dx > 0 ? 1 : 2); }
__host__ __device__ constexpr int dx_of(int j) { return j == 0 ? 0 : (j == 1 ? 1 : -1); }

// Shared memory of one plane slot, in elements E.
//   Seam s in [0, W], side UP (values with c_y = +1 from row y0 + 2s - 1) and
//   DN (c_y = -1 from row y0 + 2s), each: sigma[34], then per x slot j and c_z
//   index a value row [34]; position x' + 1 for x' in [-1, 32].
//   XH[w][side]: the halo column of warp w (side 0: x0 - 1, 1: x0 + 32; w = W
//   is written by the corner lanes and read by nobody):
//   [0, 6) c_y = 0 values, lanes (A, B) per c_z; [6, 8) sigma (A, B);
//   [8, 8 + n) c_y = +1 values of row A; [8 + n, 8 + 2n) c_y = -1 values of row B.
template <int Q, int W, typename E> struct RCfg {
    static constexpr int NPOS = 34;
    __host__ __device__ static constexpr int nzj(int j) { return nzv<Q>(dx_of(j), 1); }
    __host__ __device__ static constexpr int voff(int j, int ci)
    {
        return NPOS * (1 + (j > 0 ? nzj(0) : 0) + (j > 1 ? nzj(1) : 0) + ci);
    }
    static constexpr int SIDE = NPOS * (1 + nzv<Q>(0, 1) + 2 * nzv<Q>(1, 1));
    static constexpr int NXY = nzv<Q>(1, 1);  // c_z values of an in-plane diagonal
    static constexpr int XHW = 16;
    static constexpr int XH0 = (W + 1) * 2 * SIDE;
    static constexpr int SLOT = XH0 + (W + 1) * 2 * XHW;  // XH of warp W: the corners' spare
    static constexpr size_t SLOT_BYTES = ((size_t)SLOT * sizeof(E) + 127) / 128 * 128;
    static_assert(8 + 2 * NXY <= XHW, "halo column entry");
};

template <int Q, int ST, int W> __host__ __device__ constexpr size_t rowpair_smem()
{
    using E = typename Storage<ST>::ctype;
    using SC = tile::StageCfg<ST, W>;
    return 2 * RCfg<Q, W, E>::SLOT_BYTES + SC::NSTAGE * SC::STAGE_BYTES + 8 * SC::NSTAGE;
}

template <int Q, int ST, int W> __device__ __forceinline__ unsigned char* rp_stages(unsigned char* smem)
{
    using E = typename Storage<ST>::ctype;
    return smem + 2 * RCfg<Q, W, E>::SLOT_BYTES;
}
template <int Q, int ST, int W> __device__ __forceinline__ uint64_t* rp_barriers(unsigned char* smem)
{
    using SC = tile::StageCfg<ST, W>;
    return reinterpret_cast<uint64_t*>(rp_stages<Q, ST, W>(smem) + SC::NSTAGE * SC::STAGE_BYTES);
}
// Initialises the stage mbarriers (thread 0; the caller synchronises the block
// before the first rowpair_column).
template <int Q, int ST, int W> __device__ __forceinline__ void rp_stage_init(unsigned char* smem)
{
    if (threadIdx.x == 0) {
        uint64_t* mbar = rp_barriers<Q, ST, W>(smem);
#pragma unroll
        for (int st = 0; st < tile::StageCfg<ST, W>::NSTAGE; ++st) mbar_init(&mbar[st], 1);
        mbar_init_fence();
    }
}

// value from lane - DX (DX = +1: the lane below, -1: the lane above); the edge
// lane gets its own value back and overrides it with the halo column's
template <int DX, typename E> __device__ __forceinline__ E shfl_from(E v)
{
    if constexpr (DX > 0) return __shfl_up_sync(0xffffffffu, v, 1);
    else return __shfl_down_sync(0xffffffffu, v, 1);
}
template <int DX, typename L> __device__ __forceinline__ L shfl2_from(const L& v)
{
    return L(shfl_from<DX>(v.v.x), shfl_from<DX>(v.v.y));
}

// One tile column of one step: the tile (x0, y0) of 32 x 2W nodes, planes
// z0 <= z < z1. All 32 W threads of the block call it together (it
// synchronises). smem holds rowpair_smem<Q, ST, W>() bytes, 128-byte aligned,
// with the stage mbarriers initialised by rp_stage_init; *phase_io carries
// their phase bits from call to call. tmap views the state read as a 3D array
// of 4 nx x ny x nz values. With AMAX, amax[f] collects the largest |value|
// of field f among the nodes this thread stores. A wait for a stage that runs
// out counts one timeout in *a.timeouts; the thread then stores nothing more
// in this call and skips its later waits.
template <int Q, int ST, int W, bool AMAX>
__device__ __forceinline__ void rowpair_column(const StepArgs& a, const Scales& sc, int x0, int y0, int z0, int z1,
                                               unsigned char* smem, float (&amax)[4], const CUtensorMap* tmap,
                                               uint32_t* phase_io)
{
    using S = Storage<ST>;
    using E = typename S::ctype;
    using L = typename Lanes<E>::type;
    using C = RCfg<Q, W, E>;
    using SC = tile::StageCfg<ST, W>;
    constexpr int NC = Weights<Q>::NCLASS;
    constexpr int NPOS = C::NPOS;
    constexpr int NXY = C::NXY;
    static_assert(W >= 2 && 2 * W + 2 <= 32, "the halo rows and columns are tasks of two different warps");

    const int tid = threadIdx.x;
    const int lane = tid & 31, w = tid >> 5;
    const uint32_t nxy = (uint32_t)a.nx * (uint32_t)a.ny;
    const int gx = x0 + lane, gyA = y0 + 2 * w, gyB = gyA + 1;
    const L g0(gcomp<E>(a, 0)), g1(gcomp<E>(a, 1)), g2(gcomp<E>(a, 2));

    unsigned char* stages = rp_stages<Q, ST, W>(smem);
    uint64_t* mbar = rp_barriers<Q, ST, W>(smem);
    uint32_t phase = *phase_io;
    bool timed_out = false;

    // ---- halo roles ---------------------------------------------------------
    // row task (warp W - 1): lane A = row y0 - 1, lane B = row y0 + 2W, column x0 + lane
    // column task (warp W - 2, lanes [0, 2W + 2)): lane j < W: column x0 - 1,
    // rows of warp j; W <= j < 2W: column x0 + 32, rows of warp j - W;
    // 2W: corners at x0 - 1 (rows y0 - 1, y0 + 2W); 2W + 1: corners at x0 + 32
    const bool hrow = w == W - 1;
    const bool hcol = w == W - 2 && lane < 2 * W + 2;
    const int hj = lane;
    const bool hc_right = hcol && ((hj >= W && hj < 2 * W) || hj == 2 * W + 1);
    const bool hc_corner = hj >= 2 * W;
    const int hc_w = hj < W ? hj : hj - W;  // warp of a regular column lane
    const int hc_x = hc_right ? 32 : -1;
    // stage cells (c, r) and global positions of this thread's halo pair
    int hcA = 0, hrA = 0, hcB = 0, hrB = 0, hxA = 0, hyA = 0, hxB = 0, hyB = 0;
    if (hrow) {
        hcA = hcB = lane + SC::XOFF;
        hrA = 0;
        hrB = 2 * W + 1;
        hxA = hxB = gx;
        hyA = y0 - 1;
        hyB = y0 + 2 * W;
    } else if (hcol) {
        hcA = hcB = hc_x + SC::XOFF;
        hxA = hxB = x0 + hc_x;
        if (hc_corner) {
            hrA = 0;
            hrB = 2 * W + 1;
            hyA = y0 - 1;
            hyB = y0 + 2 * W;
        } else {
            hrA = 2 * hc_w + 1;
            hrB = 2 * hc_w + 2;
            hyA = y0 + 2 * hc_w;
            hyB = hyA + 1;
        }
    }
    const bool has_halo = hrow || hcol;
    auto in_dom = [&](int x, int y) { return x >= 0 && x < a.nx && y >= 0 && y < a.ny; };
    const bool hinA = in_dom(hxA, hyA), hinB = in_dom(hxB, hyB);
    bool hokA = false, hokB = false;
    uint32_t hxyA = 0, hxyB = 0;
    {
        int x = hxA, y = hyA;
        hokA = tile::wrap_coord(x, a.nx, a.periodic[0]) && tile::wrap_coord(y, a.ny, a.periodic[1]);
        hxyA = (uint32_t)x + (uint32_t)a.nx * (uint32_t)y;
        x = hxB;
        y = hyB;
        hokB = tile::wrap_coord(x, a.nx, a.periodic[0]) && tile::wrap_coord(y, a.ny, a.periodic[1]);
        hxyB = (uint32_t)x + (uint32_t)a.nx * (uint32_t)y;
    }

    // ---- shared-memory addressing -------------------------------------------
    auto slot_of = [&](int p) { return reinterpret_cast<E*>(smem + (size_t)((p - z0 + 1) & 1) * C::SLOT_BYTES); };
    // side base: seam s, dir 0 = UP, 1 = DN
    auto side = [&](E* sl, int s, int dir) { return sl + (s * 2 + dir) * C::SIDE; };
    auto xh = [&](E* sl, int ww, int sd) { return sl + C::XH0 + (ww * 2 + sd) * C::XHW; };

    // ---- TMA ------------------------------------------------------------------
    auto issue = [&](int p) {
        int gz = p;
        if (tid == 0 && !timed_out && tile::wrap_coord(gz, a.nz, a.periodic[2])) {
            const int st = (p - z0 + 1) % SC::NSTAGE;
            mbar_arrive_expect_tx(&mbar[st], SC::BOX_BYTES);
            tma_load_3d(stages + st * SC::STAGE_BYTES, tmap, &mbar[st], 4 * (x0 - SC::XOFF), y0 - 1, gz);
        }
    };

    // ---- register state of the z-march ----------------------------------------
    NodeAcc<L, NC> acc;
    L up_v[Q], up_s[Q];  // c_z = +1 links gathered for the next plane: value, source sigma
    L own_in[Q];         // own outgoing (., ., +1) of the previous plane
    L out[Q];            // own outgoing values of the current plane
    L sig;               // own sigma of the current plane
    bool fluidA = false, fluidB = false, fluidA_prev = false, fluidB_prev = false;
#pragma unroll
    for (int k = 0; k < Q; ++k) up_v[k] = up_s[k] = own_in[k] = L(E(0));
    acc.clear();

    // Arrival of plane p: halo exports, own outgoing values, seam exports.
    auto export_plane = [&](int p) {
        int gz = p;
        const bool zok = tile::wrap_coord(gz, a.nz, a.periodic[2]);
        const uint32_t zoff = (uint32_t)gz * nxy;
        const int st = (p - z0 + 1) % SC::NSTAGE;
        if (zok && !timed_out) {
            if (!mbar_wait_bounded(&mbar[st], (phase >> st) & 1u)) timed_out = true;
            phase ^= 1u << st;
        }
        const bool staged = zok && !timed_out;
        const unsigned char* base = stages + st * SC::STAGE_BYTES;
        auto cell = [&](int c, int r) { return base + (size_t)(r * SC::SW + c) * SC::REC; };
        E* sl = slot_of(p);

        // ---- halo tasks ------------------------------------------------------
        if (has_halo) {
            tile::Raw2<L> r;
            if (staged && hinA) S::load_at(cell(hcA, hrA), sc.inv, r.d.v.x, r.ux.v.x, r.uy.v.x, r.uz.v.x);
            else tile::load_node<ST>(a, sc, zok && hokA, zoff + hxyA, r.d.v.x, r.ux.v.x, r.uy.v.x, r.uz.v.x);
            if (staged && hinB) S::load_at(cell(hcB, hrB), sc.inv, r.d.v.y, r.ux.v.y, r.uy.v.y, r.uz.v.y);
            else tile::load_node<ST>(a, sc, zok && hokB, zoff + hxyB, r.d.v.y, r.ux.v.y, r.uy.v.y, r.uz.v.y);
            L hs;
            const NodeMoments<L> m = tile::moments_of(r, g0, g1, g2, hs);
            auto f = [&](L pv) { return feq_scaled(m.A, m.H, pv); };
            if (hrow) {
                // lane A: row y0 - 1, exports with c_y = +1 into seam 0 UP;
                // lane B: row y0 + 2W, c_y = -1 into seam W DN
                E* up = side(sl, 0, 0);
                E* dn = side(sl, W, 1);
                const L pa = m.Py * L(E(1), E(-1));
                const int pos = lane + 1;
                up[pos] = hs.v.x;
                dn[pos] = hs.v.y;
                static_for<0, 3>([&](auto jc) {
                    constexpr int j = decltype(jc)::value;
                    constexpr int dx = dx_of(j);
                    const L px = dx == 0 ? pa : (dx > 0 ? pa + m.Px : pa - m.Px);
                    static_for<0, 3>([&](auto cc) {
                        constexpr int cz = decltype(cc)::value - 1;
                        if constexpr (nzv<Q>(dx, 1) == 3 || cz == 0) {
                            constexpr int ci = czi<Q>(dx, 1, cz);
                            const L v = f(cz == 0 ? px : (cz > 0 ? px + m.Pz : px - m.Pz));
                            up[C::voff(j, ci) + pos] = v.v.x;
                            dn[C::voff(j, ci) + pos] = v.v.y;
                        }
                    });
                });
            } else {
                // column x0 - 1 exports c_x = +1, column x0 + 32 exports c_x = -1
                const int j = hc_right ? 2 : 1;
                const int pos = hc_right ? NPOS - 1 : 0;
                const L pa = m.Px * L(E(hc_right ? -1 : 1));
                const L pb = m.Py;
                const L pp = pa + pb, pm = pa - pb;
                // a corner lane writes its halo-column entries to the spare slot
                // of warp W (read by nobody), so that corner and regular lanes
                // run the same instructions
                E* x = xh(sl, hc_corner ? W : hc_w, hc_right ? 1 : 0);
                // seam targets: a regular lane's row A (c_y = -1) goes to seam hc_w DN
                // and its row B (c_y = +1) to seam hc_w + 1 UP; a corner lane's row A
                // (y0 - 1, c_y = +1) to seam 0 UP and row B (y0 + 2W, c_y = -1) to seam W DN
                E* sA = hc_corner ? side(sl, 0, 0) : side(sl, hc_w, 1);
                E* sB = hc_corner ? side(sl, W, 1) : side(sl, hc_w + 1, 0);
                sA[pos] = hs.v.x;
                sB[pos] = hs.v.y;
                x[6] = hs.v.x;
                x[7] = hs.v.y;
                static_for<0, 3>([&](auto cc) {
                    constexpr int cz = decltype(cc)::value - 1;
                    auto zt = [&](L pv) { return cz == 0 ? pv : (cz > 0 ? pv + m.Pz : pv - m.Pz); };
                    const L v0 = f(zt(pa));
                    x[2 * (cz + 1)] = v0.v.x;
                    x[2 * (cz + 1) + 1] = v0.v.y;
                    if constexpr (NXY == 3 || cz == 0) {
                        constexpr int ci = czi<Q>(1, 1, cz);
                        const L vp = f(zt(pp)), vm = f(zt(pm));
                        // a corner's row A (y0 - 1) sends c_y = +1, its row B
                        // (y0 + 2W) c_y = -1; a regular row A sends c_y = -1 and
                        // row B c_y = +1 across the seams
                        sA[C::voff(j, ci) + pos] = hc_corner ? vp.v.x : vm.v.x;
                        sB[C::voff(j, ci) + pos] = hc_corner ? vm.v.y : vp.v.y;
                        x[8 + ci] = vp.v.x;        // row A, c_y = +1: for row B of lane 0/31
                        x[8 + NXY + ci] = vm.v.y;  // row B, c_y = -1: for row A of lane 0/31
                    }
                });
            }
        }

        // ---- own nodes ---------------------------------------------------------
        tile::Raw2<L> r_own;
        if (staged) {
            S::load_at(cell(lane + SC::XOFF, 2 * w + 1), sc.inv, r_own.d.v.x, r_own.ux.v.x, r_own.uy.v.x,
                       r_own.uz.v.x);
            S::load_at(cell(lane + SC::XOFF, 2 * w + 2), sc.inv, r_own.d.v.y, r_own.ux.v.y, r_own.uy.v.y,
                       r_own.uz.v.y);
        } else {
            tile::load_node<ST>(a, sc, false, 0, r_own.d.v.x, r_own.ux.v.x, r_own.uy.v.x, r_own.uz.v.x);
            tile::load_node<ST>(a, sc, false, 0, r_own.d.v.y, r_own.ux.v.y, r_own.uy.v.y, r_own.uz.v.y);
        }
        {
            const NodeMoments<L> m = tile::moments_of(r_own, g0, g1, g2, sig);
            out[0] = m.A;
            static_for<0, (Q - 1) / 2>([&](auto ic) {
                constexpr int K = 1 + 2 * decltype(ic)::value;  // K + 1 = inv(K)
                const L pk = dir_dot<K, L>(m.Px, m.Py, m.Pz);
                const L e = fma(pk * m.H, pk, m.A);
                out[K] = e + pk;
                out[K + 1] = e - pk;
            });
        }
        fluidA = sig.v.x == E(0);
        fluidB = sig.v.y == E(0);
        // seam exports: row A sends c_y = -1 into seam w DN, row B c_y = +1 into seam w + 1 UP
        {
            E* dn = side(sl, w, 1);
            E* up = side(sl, w + 1, 0);
            const int pos = lane + 1;
            dn[pos] = sig.v.x;
            up[pos] = sig.v.y;
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                constexpr int dx = cvel(K, 0), dy = cvel(K, 1), cz = cvel(K, 2);
                if constexpr (dy == -1) dn[C::voff(jx(dx), czi<Q>(dx, dy, cz)) + pos] = out[K].v.x;
                if constexpr (dy == 1) up[C::voff(jx(dx), czi<Q>(dx, dy, cz)) + pos] = out[K].v.y;
            });
        }
        if (p + 2 <= z1) issue(p + 2);
    };

    // ---- gathers after the plane barrier ---------------------------------------
    // sigma of the in-row sources x - 1 (sgm) and x + 1 (sgp), both rows
    L sgm, sgp;
    auto row_sigmas = [&](E* sl) {
        sgm = shfl2_from<1>(sig);
        sgp = shfl2_from<-1>(sig);
        if (lane == 0) {
            const E* x = xh(sl, w, 0);
            sgm = L(x[6], x[7]);
        }
        if (lane == 31) {
            const E* x = xh(sl, w, 1);
            sgp = L(x[6], x[7]);
        }
    };
    // sigma of the source position (x - DX, y - DY) for both rows
    auto gsig = [&](E* sl, auto dxc, auto dyc) -> L {
        constexpr int DX = decltype(dxc)::value, DY = decltype(dyc)::value;
        if constexpr (DX == 0 && DY == 0) return sig;
        else if constexpr (DY == 0) return DX > 0 ? sgm : sgp;
        else if constexpr (DY == 1) {
            const E lo = side(sl, w, 0)[lane - DX + 1];
            return L(lo, DX == 0 ? sig.v.x : (DX > 0 ? sgm.v.x : sgp.v.x));
        } else {
            const E hi = side(sl, w + 1, 1)[lane - DX + 1];
            return L(DX == 0 ? sig.v.y : (DX > 0 ? sgm.v.y : sgp.v.y), hi);
        }
    };
    // value of link K arriving at rows (A, B) from the sources of the current plane
    auto gval = [&](E* sl, auto kc) -> L {
        constexpr int K = decltype(kc)::value;
        constexpr int DX = cvel(K, 0), DY = cvel(K, 1), CZ = cvel(K, 2);
        constexpr int ci = czi<Q>(DX, DY, CZ);
        constexpr int edge = DX > 0 ? 0 : 31;
        if constexpr (DX == 0 && DY == 0) return out[K];
        else if constexpr (DY == 0) {
            L v = shfl2_from<DX>(out[K]);
            if (lane == edge) {
                const E* x = xh(sl, w, DX > 0 ? 0 : 1);
                v = L(x[2 * (CZ + 1)], x[2 * (CZ + 1) + 1]);
            }
            return v;
        } else if constexpr (DY == 1) {
            const E lo = side(sl, w, 0)[C::voff(jx(DX), ci) + lane - DX + 1];
            E hi;
            if constexpr (DX == 0) hi = out[K].v.x;
            else {
                hi = shfl_from<DX>(out[K].v.x);
                if (lane == edge) hi = xh(sl, w, DX > 0 ? 0 : 1)[8 + ci];
            }
            return L(lo, hi);
        } else {
            const E hi = side(sl, w + 1, 1)[C::voff(jx(DX), ci) + lane - DX + 1];
            E lo;
            if constexpr (DX == 0) lo = out[K].v.y;
            else {
                lo = shfl_from<DX>(out[K].v.y);
                if (lane == edge) lo = xh(sl, w, DX > 0 ? 0 : 1)[8 + NXY + ci];
            }
            return L(lo, hi);
        }
    };
    auto sig_of = [&](E* sl, auto kc) -> L {
        constexpr int K = decltype(kc)::value;
        return gsig(sl, std::integral_constant<int, cvel(K, 0)>{}, std::integral_constant<int, cvel(K, 1)>{});
    };

    // c_z = -1 values of plane p complete plane p - 1, stored if it is this block's and fluid
    auto finish_prev = [&](int p, E* sl) {
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == -1) acc.template add<Q, K>(fma(sig_of(sl, kc), own_in[inv_dir(K)], gval(sl, kc)));
        });
        L d_, x_, y_, z_;
        node_finish<Q, L>(acc, d_, x_, y_, z_);
        const uint32_t zoff = (uint32_t)(p - 1) * nxy;
        if (fluidA_prev && !timed_out) {
            step_store<ST>(a.post, zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyA, d_.v.x, x_.v.x, y_.v.x,
                           z_.v.x, sc.s, a.seed);
            if constexpr (AMAX) tile::track_amax(amax, d_.v.x, x_.v.x, y_.v.x, z_.v.x);
        }
        if (fluidB_prev && !timed_out) {
            step_store<ST>(a.post, zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyB, d_.v.y, x_.v.y, y_.v.y,
                           z_.v.y, sc.s, a.seed);
            if constexpr (AMAX) tile::track_amax(amax, d_.v.y, x_.v.y, y_.v.y, z_.v.y);
        }
    };
    // plane p: the c_z = +1 links gathered last plane, then c_z = 0
    auto start_plane = [&](E* sl) {
        acc.S[0] = out[0];
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 1) acc.template add<Q, K>(fma(up_s[K], out[inv_dir(K)], up_v[K]));
        });
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 0) acc.template add<Q, K>(fma(sig_of(sl, kc), out[inv_dir(K)], gval(sl, kc)));
        });
    };
    // c_z = +1 values and sigmas of plane p wait in registers for plane p + 1,
    // and so do the own outgoing (., ., +1) values for its bounce-back
    auto carry = [&](E* sl) {
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 1) {
                up_v[K] = gval(sl, kc);
                up_s[K] = sig_of(sl, kc);
                own_in[K] = out[K];
            }
        });
    };

    issue(z0 - 1);
    issue(z0);
    // plane z0 - 1 (below the chunk): exports and carry only
    export_plane(z0 - 1);
    __syncthreads();
    {
        E* sl = slot_of(z0 - 1);
        row_sigmas(sl);
        carry(sl);
    }
    // planes of the chunk; the first finish_prev completes plane z0 - 1,
    // which is not this block's (fluid*_prev are false) and is not stored
    for (int p = z0; p < z1; ++p) {
        export_plane(p);
        __syncthreads();
        E* sl = slot_of(p);
        row_sigmas(sl);
        finish_prev(p, sl);
        start_plane(sl);
        carry(sl);
        fluidA_prev = fluidA;
        fluidB_prev = fluidB;
    }
    // plane z1 (above the chunk): its c_z = -1 values finish plane z1 - 1
    export_plane(z1);
    __syncthreads();
    {
        E* sl = slot_of(z1);
        row_sigmas(sl);
        finish_prev(z1, sl);
    }
    if (timed_out) atomicAdd(a.timeouts, 1u);
    *phase_io = phase;
}

// Tile shapes of the row-pair kernel: W warps (tile 32 x 2W), MINB resident
// blocks the register budget is sized for.
template <int Q, typename E, int V> struct RShape;
template <> struct RShape<19, float, 0> { static constexpr int W = 4, MINB = 4; };
template <> struct RShape<19, float, 1> { static constexpr int W = 8, MINB = 2; };
template <> struct RShape<19, float, 2> { static constexpr int W = 4, MINB = 3; };
template <> struct RShape<19, float, 3> { static constexpr int W = 6, MINB = 2; };
template <> struct RShape<27, float, 0> { static constexpr int W = 4, MINB = 2; };
template <> struct RShape<27, float, 1> { static constexpr int W = 8, MINB = 1; };
template <> struct RShape<27, float, 2> { static constexpr int W = 4, MINB = 3; };
template <> struct RShape<27, float, 3> { static constexpr int W = 6, MINB = 1; };
template <int V> struct RShape<19, double, V> { static constexpr int W = 4, MINB = 1; };
template <int V> struct RShape<27, double, V> { static constexpr int W = 4, MINB = 1; };
constexpr int RSHAPES = 4;

}  // namespace rp

}  // namespace lbm

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
// (B). Warp 0 computes both halo rows as one two-lane pair, warp 1 the two
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
// smem_raw holds TCfg<Q, 32, H, E>::SMEM bytes. With AMAX, amax[f] collects
// the largest |value| of field f among the nodes this thread stores.
template <int Q, int ST, int H, bool AMAX>
__device__ __forceinline__ void tile_column(const StepArgs& a, const Scales& sc, int x0, int y0, int z0, int z1,
                                            unsigned char* smem_raw, float (&amax)[4])
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

    // halo roles. Warp 0: halo rows below (lane A) and above (lane B).
    // Warp 1: halo columns, lanes 0..H+1 left (x = -1), H+2..2H+3 right (x = 32).
    const bool hrow = ty == 0;
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
    prefetch(z0 - 1);

    NodeAcc<L, NC> acc;  // plane p - 1, all but its c_z = -1 links
    L up_v[Q], up_s[Q];  // c_z = +1 links gathered for plane p: value, source sigma
    L own_in[Q];         // own outgoing (., ., +1) of plane p - 1
    bool fluidA_prev = false, fluidB_prev = false;
#pragma unroll
    for (int k = 0; k < Q; ++k) up_v[k] = up_s[k] = own_in[k] = L(E(0));
    acc.clear();

    for (int p = z0 - 1; p <= z1; ++p) {
        unsigned char* slot = smem_raw + (size_t)((p - z0 + 1) & 1) * C::SLOT_BYTES;
        V4<E>* L01 = reinterpret_cast<V4<E>*>(slot);
        V2<E>* L2 = reinterpret_cast<V2<E>*>(slot + C::L01_BYTES);
        V2<E>* DG = reinterpret_cast<V2<E>*>(slot + C::L01_BYTES + C::L2_BYTES);
        V2<E>* SG = reinterpret_cast<V2<E>*>(slot + C::L01_BYTES + C::L2_BYTES + C::DG_BYTES);

        // ---- own outgoing values (registers) and exports --------------------
        L sig;
        L out[Q];
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
        const bool fluidA = activeA && sig.v.x == E(0), fluidB = activeB && sig.v.y == E(0);
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
        if (p + 1 <= z1) prefetch(p + 1);
        __syncthreads();

        // ---- gather: c_z = -1 values finish plane p - 1 ------------------------
        if (p - 1 >= z0) {
            L dn_v[Q], dn_s[Q];
            static_for<0, NB>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                constexpr int dx = X::dx(b), dy = X::dy(b), K = kdir(dx, dy, -1);
                const int q = ppos(tx - dx, ty - dy, PW);
                const V4<E> v = L01[b * NPP + q];
                const V2<E> s = SG[q];
                dn_v[K] = L(v.x, v.y);
                dn_s[K] = L(s.x, s.y);
            });
            dn_v[KZM] = out[KZM];  // (0,0,-1): from the own node at plane p
            dn_s[KZM] = sig;
            // bounce values: own outgoing of plane p - 1 in direction inv(k) = (., ., +1)
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if constexpr (cvel(K, 2) == -1) acc.template add<K>(fma(dn_s[K], own_in[inv_dir(K)], dn_v[K]));
            });
            L d_, x_, y_, z_;
            node_finish<Q, L>(acc, d_, x_, y_, z_);
            const uint32_t zoff = (uint32_t)(p - 1) * nxy;
            if (fluidA_prev) {
                step_store<ST>(a.post, zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyA, d_.v.x, x_.v.x, y_.v.x,
                               z_.v.x, sc.s, a.seed);
                if constexpr (AMAX) track_amax(amax, d_.v.x, x_.v.x, y_.v.x, z_.v.x);
            }
            if (fluidB_prev) {
                step_store<ST>(a.post, zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyB, d_.v.y, x_.v.y, y_.v.y,
                               z_.v.y, sc.s, a.seed);
                if constexpr (AMAX) track_amax(amax, d_.v.y, x_.v.y, y_.v.y, z_.v.y);
            }
        }

        // ---- plane p: the c_z = +1 links gathered last arrival, then c_z = 0 ----
        if (p >= z0 && p < z1) {
            acc.clear();
            acc.S[0] = out[0];
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if constexpr (cvel(K, 2) == 1) acc.template add<K>(fma(up_s[K], out[inv_dir(K)], up_v[K]));
            });
            L mid_v[Q], mid_s[Q];
            static_for<0, NB>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                constexpr int dx = X::dx(b), dy = X::dy(b), K = kdir(dx, dy, 0);
                const int q = ppos(tx - dx, ty - dy, PW);
                const V4<E> v = L01[b * NPP + q];
                const V2<E> s = SG[q];
                mid_v[K] = L(v.z, v.w);
                mid_s[K] = L(s.x, s.y);
            });
            static_for<0, ND>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                constexpr int dx = X::ddx(j), dy = X::ddy(j), K = kdir(dx, dy, 0);
                const int q = ppos(tx - dx, ty - dy, PW);
                const V2<E> v = DG[j * NPP + q];
                const V2<E> s = SG[q];
                mid_v[K] = L(v.x, v.y);
                mid_s[K] = L(s.x, s.y);
            });
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if constexpr (cvel(K, 2) == 0) acc.template add<K>(fma(mid_s[K], out[inv_dir(K)], mid_v[K]));
            });
        }

        // ---- carry the c_z = +1 links of plane p + 1 -----------------------------
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int dx = X::dx(b), dy = X::dy(b), K = kdir(dx, dy, 1);
            const int q = ppos(tx - dx, ty - dy, PW);
            const V2<E> v = L2[b * NPP + q];
            const V2<E> s = SG[q];
            up_v[K] = L(v.x, v.y);
            up_s[K] = L(s.x, s.y);
        });
        up_v[KZP] = out[KZP];
        up_s[KZP] = sig;
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 1) own_in[K] = out[K];
        });
        fluidA_prev = fluidA;
        fluidB_prev = fluidB;
    }
}

// Tile-shape variants (H = half tile height, MINB = resident blocks the
// register budget is sized for). The autotuner picks one per handle
// (single box) or per batch.
template <int Q, typename E, int V> struct Shape;
template <> struct Shape<19, float, 0> { static constexpr int H = 4, MINB = 3; };
template <> struct Shape<19, float, 1> { static constexpr int H = 8, MINB = 1; };
template <> struct Shape<19, float, 2> { static constexpr int H = 8, MINB = 2; };
template <> struct Shape<19, float, 3> { static constexpr int H = 4, MINB = 4; };
template <> struct Shape<27, float, 0> { static constexpr int H = 4, MINB = 2; };
template <> struct Shape<27, float, 1> { static constexpr int H = 8, MINB = 1; };
template <> struct Shape<27, float, 2> { static constexpr int H = 2, MINB = 4; };
template <> struct Shape<27, float, 3> { static constexpr int H = 4, MINB = 3; };
template <int V> struct Shape<19, double, V> { static constexpr int H = 4, MINB = 1; };
template <int V> struct Shape<27, double, V> { static constexpr int H = 2, MINB = 1; };
constexpr int SHAPE_VARIANTS = 4;  // FP32-arithmetic formats; FP64 has one

}  // namespace tile

}  // namespace lbm

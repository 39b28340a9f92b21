// Two-node Tau1 step kernel for FP32 arithmetic (FP32, FP16 and BF16
// storage): the 2.5D z-march of tau1_tiled.cu with each thread owning two
// nodes of a tile column, (x, y) and (x, y + H), whose arithmetic runs in the
// two lanes of packed f32x2 instructions.
//
// What is computed is exactly the tiled kernel's: every node evaluates its
// outgoing equilibria once (Eq. LBMTau1, Eq. feq scaled by 1/w_k, in pairs
// k / inv(k)), exports them to shared memory per in-plane direction, and each
// destination gathers them from its 8 in-plane neighbours; walls use the
// MARKER exports and the node's own outgoing values (Algorithm "Complete
// Tau1 ... halfway bounce-back"); the velocity is multiplied once by 1/rho
// (Algorithm "Optimized Tau1 ... stores velocity"). Lane by lane the
// operations and their order are those of the tiled kernel, so both give the
// same bits.
//
// Tile = 32 x 2H nodes, block = 32 x H threads. Shared memory is indexed by
// "pair positions" (x', y'), x' in [-1, 32], y' in [-1, H]: lane A holds tile
// node (x', y'), lane B node (x', y' + H). A thread at (x, y) then finds both
// of its sources x - c_k at pair position (x - c_x, y - c_y). Pair row -1
// holds the halo row below (lane A) and interior row H-1 (lane B); pair row H
// holds interior row H (lane A) and the halo row above (lane B). Warp 0
// computes both halo rows as one packed pair, warp 1 the halo columns; the
// owners of rows H-1 and H copy their exports into pair rows -1 and H.
//
// Per slot, each exchange block b stores float4 {c_z=-1: A, B; c_z=0: A, B}
// and float2 {c_z=+1: A, B}; D3Q19's in-plane diagonals are float2 {A, B}.
#include "kernels.h"
#include "pack2.cuh"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

constexpr unsigned MARKER_BITS = 0x7FBADBADu;  // NaN payload arithmetic never produces
__device__ __forceinline__ float marker() { return __uint_as_float(MARKER_BITS); }
__device__ __forceinline__ bool is_marker(float v) { return __float_as_uint(v) == MARKER_BITS; }

__host__ __device__ constexpr int kdir(int cx, int cy, int cz)
{
    for (int k = 0; k < 27; ++k)
        if (cvel(k, 0) == cx && cvel(k, 1) == cy && cvel(k, 2) == cz) return k;
    return -1;
}

// Exchange blocks (in-plane direction of block b) and D3Q19 diagonal slots.
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

template <int Q, int TX, int H> struct PCfg {
    static constexpr int NB = Xch<Q>::NB, ND = Xch<Q>::ND;
    static constexpr int PW = TX + 2;
    static constexpr int NPP = (TX + 2) * (H + 2);  // pair positions
    static constexpr int NT = TX * H;
    // slot layout: L01[NB][NPP] float4 | L2[NB][NPP] float2 | DG[ND][NPP] float2
    static constexpr size_t L01_BYTES = (size_t)NB * NPP * sizeof(float4);
    static constexpr size_t L2_BYTES = (size_t)NB * NPP * sizeof(float2);
    static constexpr size_t SLOT_BYTES = L01_BYTES + L2_BYTES + (size_t)ND * NPP * sizeof(float2);
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
struct Raw2 {
    f2 d, ux, uy, uz;
    int flagA, flagB;
};

template <int ST>
__device__ __forceinline__ void load_one(const StepArgs& a, bool ok, uint32_t i, float& d, float& ux, float& uy,
                                         float& uz, int& flag)
{
    using S = Storage<ST>;
    using st = typename S::stype;
    flag = FLAG_SOLID;
    d = ux = uy = uz = 0.f;
    if (!ok) return;
    flag = __ldg(a.flags + i);
    d = S::load(static_cast<const st*>(a.pre[0]), i, a.inv_scale[0]);
    ux = S::load(static_cast<const st*>(a.pre[1]), i, a.inv_scale[1]);
    uy = S::load(static_cast<const st*>(a.pre[2]), i, a.inv_scale[2]);
    uz = S::load(static_cast<const st*>(a.pre[3]), i, a.inv_scale[3]);
}

template <int ST>
__device__ __forceinline__ void load_pair(const StepArgs& a, bool okA, uint32_t iA, bool okB, uint32_t iB, Raw2& r)
{
    load_one<ST>(a, okA, iA, r.d.v.x, r.ux.v.x, r.uy.v.x, r.uz.v.x, r.flagA);
    load_one<ST>(a, okB, iB, r.d.v.y, r.ux.v.y, r.uy.v.y, r.uz.v.y, r.flagB);
}

__device__ __forceinline__ NodeMoments<f2> moments2(const Raw2& r, const StepArgs& a)
{
    return node_moments<f2>(r.d, r.ux, r.uy, r.uz, f2(a.gf[0]), f2(a.gf[1]), f2(a.gf[2]));
}

// Replace lanes of solid (or outside) nodes by MARKER.
__device__ __forceinline__ f2 mark(f2 v, bool sA, bool sB)
{
    return f2(sA ? marker() : v.v.x, sB ? marker() : v.v.y);
}

template <int Q, int ST, int TX, int H, int MINB>
__global__ void __launch_bounds__(TX * H, MINB) tau1_pair_kernel(StepArgs a, int ntx, int ntiles, int chunk)
{
    using C = PCfg<Q, TX, H>;
    using S = Storage<ST>;
    using st = typename S::stype;
    using X = Xch<Q>;
    constexpr int NPP = C::NPP, PW = C::PW, NB = C::NB, ND = C::ND;
    constexpr int NC = Weights<Q>::NCLASS;
    constexpr int KZP = kdir(0, 0, 1), KZM = kdir(0, 0, -1);
    constexpr int TY = 2 * H;

    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;  // pair row = warp index
    const int my = ppos(tx, ty, PW);

    const int tile = blockIdx.x % ntiles;
    const int z0 = (blockIdx.x / ntiles) * chunk;
    const int z1 = min(a.nz, z0 + chunk);
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    const uint32_t nxy = (uint32_t)a.nx * (uint32_t)a.ny;
    const int gx = x0 + tx, gyA = y0 + ty, gyB = y0 + ty + H;
    const bool activeA = gx < a.nx && gyA < a.ny;
    const bool activeB = gx < a.nx && gyB < a.ny;

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
    const int hcs = tx < H + 2 ? 1 : -1;                  // column ring: exports with dx = hcs
    const int hctx = tx < H + 2 ? -1 : TX;
    const int hcty = tx < H + 2 ? tx - 1 : tx - (H + 2) - 1;  // pair row of the column slot
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
    const int hc_b0 = hcs > 0 ? 0 : 1;  // block of (hcs, 0)
    const int hc_bp = (Q == 27) ? (hcs > 0 ? block_of(1, 1) : block_of(-1, 1)) : (hcs > 0 ? diag_of(1, 1) : diag_of(-1, 1));
    const int hc_bm = (Q == 27) ? (hcs > 0 ? block_of(1, -1) : block_of(-1, -1)) : (hcs > 0 ? diag_of(1, -1) : diag_of(-1, -1));

    Raw2 r_own, r_halo;
    auto prefetch = [&](int p) {
        int gz = p;
        const bool zok = wrap_coord(gz, a.nz, a.periodic[2]);
        const uint32_t zoff = (uint32_t)gz * nxy;
        load_pair<ST>(a, zok && okA, zoff + xyA, zok && okB, zoff + xyB, r_own);
        if (has_halo) load_pair<ST>(a, zok && hokA, zoff + hxyA, zok && hokB, zoff + hxyB, r_halo);
    };
    prefetch(z0 - 1);

    NodeAcc<f2, NC> acc;  // plane p - 1, all but its c_z = -1 links
    f2 up_in[Q];          // c_z = +1 links gathered for plane p
    f2 own_in[Q];         // own outgoing (., ., +1) of plane p - 1
    int flagA_prev = FLAG_SOLID, flagB_prev = FLAG_SOLID;
#pragma unroll
    for (int k = 0; k < Q; ++k) up_in[k] = own_in[k] = f2(0.f);
    acc.clear();

    for (int p = z0 - 1; p <= z1; ++p) {
        unsigned char* slot = smem_raw + (size_t)((p - z0 + 1) & 1) * C::SLOT_BYTES;
        float4* L01 = reinterpret_cast<float4*>(slot);
        float2* L2 = reinterpret_cast<float2*>(slot + C::L01_BYTES);
        float2* DG = reinterpret_cast<float2*>(slot + C::L01_BYTES + C::L2_BYTES);

        // ---- own outgoing values (registers) and exports ------------------
        const Raw2 cur = r_own;
        const bool sA = cur.flagA & FLAG_SOLID, sB = cur.flagB & FLAG_SOLID;
        f2 out[Q];
        {
            const NodeMoments<f2> m = moments2(cur, a);
            out[0] = m.A;
            static_for<0, (Q - 1) / 2>([&](auto ic) {
                constexpr int K = 1 + 2 * decltype(ic)::value;  // K + 1 = inv(K)
                const f2 pk = dir_dot<K, f2>(m.Px, m.Py, m.Pz);
                const f2 e = fma(pk * m.H, pk, m.A);
                out[K] = e + pk;
                out[K + 1] = e - pk;
            });
            if (__any_sync(0xffffffffu, sA || sB)) {
#pragma unroll
                for (int k = 0; k < Q; ++k) out[k] = mark(out[k], sA, sB);
            }
        }
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int dx = X::dx(b), dy = X::dy(b);
            const f2 vm = out[kdir(dx, dy, -1)], v0 = out[kdir(dx, dy, 0)], vp = out[kdir(dx, dy, 1)];
            L01[b * NPP + my] = make_float4(vm.v.x, vm.v.y, v0.v.x, v0.v.y);
            L2[b * NPP + my] = vp.v;
        });
        static_for<0, ND>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            DG[j * NPP + my] = out[kdir(X::ddx(j), X::ddy(j), 0)].v;
        });
        // interior rows H-1 and H also appear in pair rows -1 (lane B) and H (lane A)
        if (ty == H - 1) {
            const int q = ppos(tx, -1, PW);
            static_for<0, NB>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                if constexpr (X::dy(b) == 1) {
                    float* l01 = reinterpret_cast<float*>(&L01[b * NPP + q]);
                    l01[1] = out[kdir(X::dx(b), 1, -1)].v.x;
                    l01[3] = out[kdir(X::dx(b), 1, 0)].v.x;
                    reinterpret_cast<float*>(&L2[b * NPP + q])[1] = out[kdir(X::dx(b), 1, 1)].v.x;
                }
            });
            static_for<0, ND>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                if constexpr (X::ddy(j) == 1) reinterpret_cast<float*>(&DG[j * NPP + q])[1] = out[kdir(X::ddx(j), 1, 0)].v.x;
            });
        }
        if (ty == 0) {
            const int q = ppos(tx, H, PW);
            static_for<0, NB>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                if constexpr (X::dy(b) == -1) {
                    float* l01 = reinterpret_cast<float*>(&L01[b * NPP + q]);
                    l01[0] = out[kdir(X::dx(b), -1, -1)].v.y;
                    l01[2] = out[kdir(X::dx(b), -1, 0)].v.y;
                    reinterpret_cast<float*>(&L2[b * NPP + q])[0] = out[kdir(X::dx(b), -1, 1)].v.y;
                }
            });
            static_for<0, ND>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                if constexpr (X::ddy(j) == -1) reinterpret_cast<float*>(&DG[j * NPP + q])[0] = out[kdir(X::ddx(j), -1, 0)].v.y;
            });
        }

        // ---- halo exports ---------------------------------------------------
        if (hrow) {
            // lane A: row below, exports with dy = +1; lane B: row above, dy = -1
            const NodeMoments<f2> m = moments2(r_halo, a);
            const bool hsA = r_halo.flagA & FLAG_SOLID, hsB = r_halo.flagB & FLAG_SOLID;
            const f2 pa = m.Py * f2(1.f, -1.f);
            const f2 pb = m.Px;
            auto f = [&](f2 pv) { return mark(feq_scaled(m.A, m.H, pv), hsA, hsB); };
            const int qA = ppos(tx, -1, PW), qB = ppos(tx, H, PW);
            auto put_block = [&](int bA, int bB, f2 vm, f2 v0, f2 vp) {
                float* la = reinterpret_cast<float*>(&L01[bA * NPP + qA]);
                la[0] = vm.v.x;
                la[2] = v0.v.x;
                reinterpret_cast<float*>(&L2[bA * NPP + qA])[0] = vp.v.x;
                float* lb = reinterpret_cast<float*>(&L01[bB * NPP + qB]);
                lb[1] = vm.v.y;
                lb[3] = v0.v.y;
                reinterpret_cast<float*>(&L2[bB * NPP + qB])[1] = vp.v.y;
            };
            put_block(block_of(0, 1), block_of(0, -1), f(pa - m.Pz), f(pa), f(pa + m.Pz));
            const f2 pp = pa + pb, pm = pa - pb;
            if constexpr (Q == 27) {
                put_block(block_of(1, 1), block_of(1, -1), f(pp - m.Pz), f(pp), f(pp + m.Pz));
                put_block(block_of(-1, 1), block_of(-1, -1), f(pm - m.Pz), f(pm), f(pm + m.Pz));
            } else {
                const f2 vpp = f(pp), vpm = f(pm);
                reinterpret_cast<float*>(&DG[diag_of(1, 1) * NPP + qA])[0] = vpp.v.x;
                reinterpret_cast<float*>(&DG[diag_of(1, -1) * NPP + qB])[1] = vpp.v.y;
                reinterpret_cast<float*>(&DG[diag_of(-1, 1) * NPP + qA])[0] = vpm.v.x;
                reinterpret_cast<float*>(&DG[diag_of(-1, -1) * NPP + qB])[1] = vpm.v.y;
            }
        } else if (hcol) {
            // both lanes exports with dx = hcs
            const NodeMoments<f2> m = moments2(r_halo, a);
            const bool hsA = r_halo.flagA & FLAG_SOLID, hsB = r_halo.flagB & FLAG_SOLID;
            const f2 pa = m.Px * f2((float)hcs);
            const f2 pb = m.Py;
            auto f = [&](f2 pv) { return mark(feq_scaled(m.A, m.H, pv), hsA, hsB); };
            auto put_block = [&](int b, f2 vm, f2 v0, f2 vp) {
                L01[b * NPP + hc_pos] = make_float4(vm.v.x, vm.v.y, v0.v.x, v0.v.y);
                L2[b * NPP + hc_pos] = vp.v;
            };
            put_block(hc_b0, f(pa - m.Pz), f(pa), f(pa + m.Pz));
            const f2 pp = pa + pb, pm = pa - pb;
            if constexpr (Q == 27) {
                put_block(hc_bp, f(pp - m.Pz), f(pp), f(pp + m.Pz));
                put_block(hc_bm, f(pm - m.Pz), f(pm), f(pm + m.Pz));
            } else {
                DG[hc_bp * NPP + hc_pos] = f(pp).v;
                DG[hc_bm * NPP + hc_pos] = f(pm).v;
            }
        }
        if (p + 1 <= z1) prefetch(p + 1);
        __syncthreads();

        // ---- gather ---------------------------------------------------------
        f2 dn[Q], mid[Q], up_out[Q];  // c_z = -1 (plane p-1), 0 (plane p), +1 (plane p+1)
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int dx = X::dx(b), dy = X::dy(b);
            const int q = ppos(tx - dx, ty - dy, PW);
            const float4 v = L01[b * NPP + q];
            const float2 w = L2[b * NPP + q];
            dn[kdir(dx, dy, -1)] = f2(v.x, v.y);
            mid[kdir(dx, dy, 0)] = f2(v.z, v.w);
            up_out[kdir(dx, dy, 1)] = f2(w);
        });
        static_for<0, ND>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            constexpr int dx = X::ddx(j), dy = X::ddy(j);
            mid[kdir(dx, dy, 0)] = f2(DG[j * NPP + ppos(tx - dx, ty - dy, PW)]);
        });
        dn[KZM] = out[KZM];
        up_out[KZP] = out[KZP];

        // ---- plane p - 1: its c_z = -1 links, then finish ---------------------
        if (p - 1 >= z0) {
            const bool fluidA = activeA && !(flagA_prev & FLAG_SOLID);
            const bool fluidB = activeB && !(flagB_prev & FLAG_SOLID);
            const bool wall = (fluidA && (flagA_prev & FLAG_WALL_LINK)) || (fluidB && (flagB_prev & FLAG_WALL_LINK));
            if (__any_sync(0xffffffffu, wall)) {
                static_for<1, Q>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    if constexpr (cvel(K, 2) == -1) {
                        const f2 bb = own_in[inv_dir(K)];
                        dn[K] = f2(is_marker(dn[K].v.x) ? bb.v.x : dn[K].v.x, is_marker(dn[K].v.y) ? bb.v.y : dn[K].v.y);
                    }
                });
            }
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if constexpr (cvel(K, 2) == -1) acc.template add<K>(dn[K]);
            });
            f2 dd, ux, uy, uz;
            node_finish<Q, f2>(acc, dd, ux, uy, uz);
            const uint32_t zoff = (uint32_t)(p - 1) * nxy;
            if (fluidA) {
                const uint32_t i = zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyA;
                S::store(static_cast<st*>(a.post[0]), i, dd.v.x, a.scale[0]);
                S::store(static_cast<st*>(a.post[1]), i, ux.v.x, a.scale[1]);
                S::store(static_cast<st*>(a.post[2]), i, uy.v.x, a.scale[2]);
                S::store(static_cast<st*>(a.post[3]), i, uz.v.x, a.scale[3]);
            }
            if (fluidB) {
                const uint32_t i = zoff + (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gyB;
                S::store(static_cast<st*>(a.post[0]), i, dd.v.y, a.scale[0]);
                S::store(static_cast<st*>(a.post[1]), i, ux.v.y, a.scale[1]);
                S::store(static_cast<st*>(a.post[2]), i, uy.v.y, a.scale[2]);
                S::store(static_cast<st*>(a.post[3]), i, uz.v.y, a.scale[3]);
            }
        }

        // ---- plane p: c_z = +1 links (last arrival) and c_z = 0 links ------
        if (p >= z0 && p < z1) {
            const bool fluidA = activeA && !sA, fluidB = activeB && !sB;
            const bool wall = (fluidA && (cur.flagA & FLAG_WALL_LINK)) || (fluidB && (cur.flagB & FLAG_WALL_LINK));
            if (__any_sync(0xffffffffu, wall)) {
                static_for<1, Q>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    const f2 bb = out[inv_dir(K)];
                    if constexpr (cvel(K, 2) == 1) {
                        up_in[K] = f2(is_marker(up_in[K].v.x) ? bb.v.x : up_in[K].v.x,
                                      is_marker(up_in[K].v.y) ? bb.v.y : up_in[K].v.y);
                    } else if constexpr (cvel(K, 2) == 0) {
                        mid[K] = f2(is_marker(mid[K].v.x) ? bb.v.x : mid[K].v.x, is_marker(mid[K].v.y) ? bb.v.y : mid[K].v.y);
                    }
                });
            }
            acc.clear();
            acc.S[0] = out[0];
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if constexpr (cvel(K, 2) == 1) acc.template add<K>(up_in[K]);
            });
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if constexpr (cvel(K, 2) == 0) acc.template add<K>(mid[K]);
            });
        }
        // ---- carry ------------------------------------------------------------
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 1) {
                up_in[K] = up_out[K];
                own_in[K] = out[K];
            }
        });
        flagA_prev = cur.flagA;
        flagB_prev = cur.flagB;
    }
}

// Tile-shape variants (H = half tile height, MINB = resident blocks the
// register budget is sized for). The autotuner picks one per handle.
template <int Q, int V> struct PairShape;
template <> struct PairShape<19, 0> { static constexpr int H = 8, MINB = 1; };
template <> struct PairShape<19, 1> { static constexpr int H = 4, MINB = 3; };
template <> struct PairShape<19, 2> { static constexpr int H = 8, MINB = 2; };
template <> struct PairShape<27, 0> { static constexpr int H = 4, MINB = 2; };
template <> struct PairShape<27, 1> { static constexpr int H = 8, MINB = 1; };
template <> struct PairShape<27, 2> { static constexpr int H = 4, MINB = 1; };
constexpr int PAIR_VARIANTS = 3;

template <int Q, int ST, int V>
cudaError_t launch_pair_t(const StepArgs& a, cudaStream_t s)
{
    constexpr int TX = 32, H = PairShape<Q, V>::H;
    using C = PCfg<Q, TX, H>;
    auto kern = tau1_pair_kernel<Q, ST, TX, H, PairShape<Q, V>::MINB>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int ntx = (a.nx + TX - 1) / TX;
    const int nty = (a.ny + 2 * H - 1) / (2 * H);
    const int ntiles = ntx * nty;
    const int chunk = a.nz < 32 ? a.nz : 32;
    const int nchunks = (a.nz + chunk - 1) / chunk;
    const long long blocks = (long long)ntiles * nchunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, C::NT, C::SMEM, s>>>(a, ntx, ntiles, chunk);
    return cudaGetLastError();
}

template <int Q, int ST>
cudaError_t launch_pair_v(int variant, const StepArgs& a, cudaStream_t s)
{
    switch (variant) {
    case 0: return launch_pair_t<Q, ST, 0>(a, s);
    case 1: return launch_pair_t<Q, ST, 1>(a, s);
    case 2: return launch_pair_t<Q, ST, 2>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool tau1_pair_supported(int q, int storage, int64_t n)
{
    return (q == 19 || q == 27) && storage >= ST_F32 && storage <= ST_BF16S && n > 0 && n < ((int64_t)1 << 31);
}

int tau1_pair_variants(int) { return PAIR_VARIANTS; }

cudaError_t launch_tau1_pair(int q, int storage, int variant, const StepArgs& a, cudaStream_t s)
{
    switch (q * 10 + storage) {
    case 190 + ST_F32: return launch_pair_v<19, ST_F32>(variant, a, s);
    case 190 + ST_F16S: return launch_pair_v<19, ST_F16S>(variant, a, s);
    case 190 + ST_BF16S: return launch_pair_v<19, ST_BF16S>(variant, a, s);
    case 270 + ST_F32: return launch_pair_v<27, ST_F32>(variant, a, s);
    case 270 + ST_F16S: return launch_pair_v<27, ST_F16S>(variant, a, s);
    case 270 + ST_BF16S: return launch_pair_v<27, ST_BF16S>(variant, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

// Tiled Tau1 step kernel: 2.5D z-march with shared-memory exchange of the
// equilibria each node sends to its in-plane neighbours.
//
// Tau1 (Eq. LBMTau1) says the population arriving at x along c_k is
// f_k^eq of the source x - c_k. Each node therefore evaluates its q outgoing
// equilibria once (Eq. feq, scaled by 1/w_k, as pairs k / inv(k) that share
// one fma chain) and every destination only gathers and adds. This is the
// buffering of neighbour data inside the processor that the paper's
// complexity analysis (Section 2.1.3) asks for, so that HBM sees one read and
// one write of (rho, u) per node.
//
// Block = TX x TY threads = one tile of an x-y plane (a warp is one tile row)
// marching over planes z0..z1-1. At the "arrival" of plane p every tile
// position computes its outgoing values; for each in-plane direction
// (dx, dy) != 0 it stores the 4-vector {c_z = -1, 0, +1, unused} in slot
// p % 2 of shared memory (D3Q19's four in-plane diagonals, which only exist
// with c_z = 0, go to four scalar arrays instead). The one-node ring around
// the tile exports only the directions that point into the tile. After one
// barrier each thread gathers from its 8 in-plane neighbours: the c_z = -1
// components complete destination plane p-1, c_z = 0 components go into
// plane p, and c_z = +1 components wait one arrival in registers. The
// (0,0,+-1) links and the rest direction never leave the thread.
//
// Walls (Algorithm "Complete Tau1 ... halfway bounce-back"): a solid node, or
// a position beyond a non-periodic face, exports a NaN payload (MARKER) that
// arithmetic never produces. For a warp that holds a node with a wall link,
// each MARKER is replaced by the node's own outgoing value in direction
// inv(k) of the destination plane: for plane p it is in registers; for the
// c_z = -1 links of plane p-1 the needed own values (directions (., ., +1))
// were kept from the previous arrival. Other warps add without checks.
//
// Grid: one block per (z-chunk, tile), ordered chunk-major, so the tiles of a
// chunk run side by side and each tile's halo reads hit L2.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

template <typename T> struct __align__(4 * sizeof(T)) V4 {
    T x, y, z, w;
};

template <typename T> struct Marker;
template <> struct Marker<float> {
    static constexpr unsigned BITS = 0x7FBADBADu;
    __device__ static __forceinline__ float value() { return __uint_as_float(BITS); }
    __device__ static __forceinline__ bool is(float v) { return __float_as_uint(v) == BITS; }
};
template <> struct Marker<double> {
    static constexpr unsigned long long BITS = 0x7FF4BADBADBADBADull;
    __device__ static __forceinline__ double value() { return __longlong_as_double((long long)BITS); }
    __device__ static __forceinline__ bool is(double v) { return (unsigned long long)__double_as_longlong(v) == BITS; }
};

// Direction index of velocity (cx, cy, cz), or -1.
__host__ __device__ constexpr int kdir(int cx, int cy, int cz)
{
    for (int k = 0; k < 27; ++k)
        if (cvel(k, 0) == cx && cvel(k, 1) == cy && cvel(k, 2) == cz) return k;
    return -1;
}

// Exchange layout. Block b carries in-plane direction (dx(b), dy(b)) with
// lanes c_z = -1, 0, +1. D3Q19 has 4 face blocks plus 4 diagonal scalars
// (diagonal j = in-plane direction (ddx(j), ddy(j)), c_z = 0).
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

// Raw state of one node as loaded from global memory.
template <typename T> struct Raw {
    T d, ux, uy, uz;
    int flag;  // node flags; FLAG_SOLID also for positions beyond a non-periodic face
};

template <int Q, int ST, int TX, int TY> struct Cfg {
    using S = Storage<ST>;
    using T = typename S::ctype;
    using st = typename S::stype;
    static constexpr int NB = Xch<Q>::NB, ND = Xch<Q>::ND;
    static constexpr int PW = TX + 2;
    static constexpr int NPOS = (TX + 2) * (TY + 2);
    static constexpr int NHALO = 2 * TX + 2 * (TY + 2);
    static constexpr int NT = TX * TY;
    static constexpr int NSLOT = 2;
    static constexpr size_t SLOT_BYTES = (size_t)NPOS * (NB * sizeof(V4<T>) + ND * sizeof(T));
    static constexpr size_t SMEM = NSLOT * SLOT_BYTES;
    static_assert(NHALO <= NT, "the halo ring must fit one position per thread");
    static_assert(TX == 32, "a warp is one tile row");
};

__device__ __forceinline__ int pos_of(int tx, int ty, int pw) { return (ty + 1) * pw + (tx + 1); }

// Wraps c on a periodic axis; false if it lies beyond a non-periodic face.
__device__ __forceinline__ bool wrap_coord(int& c, int n, int periodic)
{
    if (c >= 0 && c < n) return true;
    if (!periodic) return false;
    c %= n;
    if (c < 0) c += n;
    return true;
}

// Loads the raw state of node i (ok = inside the box after wrapping).
template <int ST, typename T>
__device__ __forceinline__ void load_raw(const StepArgs& a, bool ok, uint32_t i, Raw<T>& r)
{
    using S = Storage<ST>;
    using st = typename S::stype;
    r.flag = FLAG_SOLID;
    r.d = r.ux = r.uy = r.uz = T(0);
    if (!ok) return;
    // the five loads are issued together (no dependence on the flag)
    r.flag = __ldg(a.flags + i);
    r.d = S::load(static_cast<const st*>(a.pre[0]), i, a.inv_scale[0]);
    r.ux = S::load(static_cast<const st*>(a.pre[1]), i, a.inv_scale[1]);
    r.uy = S::load(static_cast<const st*>(a.pre[2]), i, a.inv_scale[2]);
    r.uz = S::load(static_cast<const st*>(a.pre[3]), i, a.inv_scale[3]);
}

// Exchange block of in-plane direction (dx, dy), D3Q27 numbering, and the
// D3Q19 diagonal slot of (dx, dy) (both at run time, evaluated once per thread).
__device__ __forceinline__ int block_of(int dx, int dy)
{
    if (dy == 0) return dx > 0 ? 0 : 1;
    if (dx == 0) return dy > 0 ? 2 : 3;
    if (dx == dy) return dx > 0 ? 4 : 5;
    return dx > 0 ? 6 : 7;
}
__device__ __forceinline__ int diag_of(int dx, int dy)
{
    if (dx == dy) return dx > 0 ? 0 : 1;
    return dx > 0 ? 3 : 2;
}

// Where a halo-ring node stores its exports: only the in-plane directions
// pointing into the tile. Row ring: directions (db, s) with db = 0, +1, -1;
// column ring: (s, db). off0 is the block of db = 0; offp / offm the blocks
// (D3Q27) or diagonal slots (D3Q19) of db = +1 / -1, as element offsets
// within their arrays.
struct HaloPlan {
    int off0, offp, offm;
    bool col;  // column ring (normal along x)
    float sgn; // s as a multiplier (exact)
};

template <int Q, int NPOS>
__device__ __forceinline__ HaloPlan halo_plan(bool col, int s, int pos)
{
    HaloPlan h;
    h.col = col;
    h.sgn = (float)s;
    auto dxy = [&](int db, int& dx, int& dy) {
        if (col) { dx = s; dy = db; } else { dx = db; dy = s; }
    };
    int dx, dy;
    dxy(0, dx, dy);
    h.off0 = block_of(dx, dy) * NPOS + pos;
    dxy(1, dx, dy);
    h.offp = (Q == 27 ? block_of(dx, dy) : diag_of(dx, dy)) * NPOS + pos;
    dxy(-1, dx, dy);
    h.offm = (Q == 27 ? block_of(dx, dy) : diag_of(dx, dy)) * NPOS + pos;
    return h;
}

// Exports of a halo-ring node. The values are bitwise those its own tile
// computes for the same directions (same p, same fma chain).
template <int Q, typename T>
__device__ __forceinline__ void store_halo_exports(V4<T>* side, T* diag, const HaloPlan& h, const Raw<T>& r,
                                                   const StepArgs& a)
{
    const NodeMoments<T> m = node_moments<T>(r.d, r.ux, r.uy, r.uz, gcomp<T>(a, 0), gcomp<T>(a, 1), gcomp<T>(a, 2));
    const T pa = T(h.sgn) * (h.col ? m.Px : m.Py);  // along the ring normal
    const T pb = h.col ? m.Py : m.Px;               // perpendicular, in-plane
    const bool solid = r.flag & FLAG_SOLID;
    const T M = Marker<T>::value();
    auto f = [&](T p) { return solid ? M : feq_scaled(m.A, m.H, p); };
    side[h.off0] = V4<T>{f(pa - m.Pz), f(pa), f(pa + m.Pz), T(0)};
    if constexpr (Q == 27) {
        const T pp = pa + pb, pm = pa - pb;
        side[h.offp] = V4<T>{f(pp - m.Pz), f(pp), f(pp + m.Pz), T(0)};
        side[h.offm] = V4<T>{f(pm - m.Pz), f(pm), f(pm + m.Pz), T(0)};
    } else {
        diag[h.offp] = f(pa + pb);
        diag[h.offm] = f(pa - pb);
    }
}

template <int Q, int ST, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB) tau1_tiled_kernel(StepArgs a, int ntx, int ntiles, int chunk)
{
    using C = Cfg<Q, ST, TX, TY>;
    using T = typename C::T;
    using st = typename C::st;
    using S = typename C::S;
    using X = Xch<Q>;
    constexpr int NPOS = C::NPOS, PW = C::PW, NB = C::NB, ND = C::ND;
    constexpr int NC = Weights<Q>::NCLASS;
    constexpr int KZP = kdir(0, 0, 1), KZM = kdir(0, 0, -1);

    extern __shared__ __align__(32) unsigned char smem_raw[];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;  // a warp is one tile row: ty = warp index
    const int my_pos = pos_of(tx, ty, PW);
    // halo ring: warp 0 the row y = -1, warp 1 the row y = TY, warp 2 both
    // columns (lanes 0..TY+1 at x = -1, lanes TY+2..2TY+3 at x = TX)
    int hmode = -1, hs = 0, htx = 0, hty = 0;
    if (ty == 0) { hmode = 0; hs = 1; htx = tx; hty = -1; }
    else if (ty == 1) { hmode = 0; hs = -1; htx = tx; hty = TY; }
    else if (ty == 2 && tx < TY + 2) { hmode = 1; hs = 1; htx = -1; hty = tx - 1; }
    else if (ty == 2 && tx < 2 * (TY + 2)) { hmode = 1; hs = -1; htx = TX; hty = tx - (TY + 2) - 1; }
    const HaloPlan hplan = halo_plan<Q, NPOS>(hmode == 1, hs, pos_of(htx, hty, PW));

    const int tile = blockIdx.x % ntiles;
    const int z0 = (blockIdx.x / ntiles) * chunk;
    const int z1 = min(a.nz, z0 + chunk);
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < a.nx && gy < a.ny;
    const uint32_t nxy = (uint32_t)a.nx * (uint32_t)a.ny;

    // in-plane offsets of the own and halo positions (wrapped once)
    int wx = gx, wy = gy;
    const bool own_xy_ok = wrap_coord(wx, a.nx, a.periodic[0]) && wrap_coord(wy, a.ny, a.periodic[1]);
    const uint32_t own_xy = (uint32_t)wx + (uint32_t)a.nx * (uint32_t)wy;
    int hx = x0 + htx, hy = y0 + hty;
    const bool halo_xy_ok = hmode >= 0 && wrap_coord(hx, a.nx, a.periodic[0]) && wrap_coord(hy, a.ny, a.periodic[1]);
    const uint32_t halo_xy = (uint32_t)hx + (uint32_t)a.nx * (uint32_t)hy;
    const uint32_t out_xy = (uint32_t)gx + (uint32_t)a.nx * (uint32_t)gy;  // stores (active nodes only)

    Raw<T> r_own, r_halo;
    auto prefetch = [&](int p) {
        int gz = p;
        const bool zok = wrap_coord(gz, a.nz, a.periodic[2]);
        const uint32_t zoff = (uint32_t)gz * nxy;
        load_raw<ST>(a, zok && own_xy_ok, zoff + own_xy, r_own);
        if (hmode >= 0) load_raw<ST>(a, zok && halo_xy_ok, zoff + halo_xy, r_halo);
    };
    prefetch(z0 - 1);

    NodeAcc<T, NC> acc;          // plane p - 1, all but its c_z = -1 links
    int flag_prev = FLAG_SOLID;  // own node flags at plane p - 1
    T up_in[Q];   // c_z = +1 link values gathered for plane p (by k)
    T own_in[Q];  // own outgoing (., ., +1) of plane p - 1: bounce values of its c_z = -1 links
#pragma unroll
    for (int k = 0; k < Q; ++k) up_in[k] = own_in[k] = T(0);
    acc.clear();

    for (int p = z0 - 1; p <= z1; ++p) {
        unsigned char* slot = smem_raw + (size_t)((p - z0 + 1) & 1) * C::SLOT_BYTES;
        V4<T>* side = reinterpret_cast<V4<T>*>(slot);
        T* diag = reinterpret_cast<T*>(slot + (size_t)NPOS * NB * sizeof(V4<T>));

        // own outgoing values (kept in registers) and their exports
        const Raw<T> cur = r_own;
        T out[Q];
        {
            const NodeMoments<T> m =
                node_moments<T>(cur.d, cur.ux, cur.uy, cur.uz, gcomp<T>(a, 0), gcomp<T>(a, 1), gcomp<T>(a, 2));
            out[0] = m.A;
            static_for<0, (Q - 1) / 2>([&](auto ic) {
                constexpr int K = 1 + 2 * decltype(ic)::value;  // K + 1 = inv(K)
                const T pk = dir_dot<K, T>(m.Px, m.Py, m.Pz);
                const T e = fma(pk * m.H, pk, m.A);
                out[K] = e + pk;
                out[K + 1] = e - pk;
            });
            const bool solid = cur.flag & FLAG_SOLID;
            if (__any_sync(0xffffffffu, solid)) {
                const T M = Marker<T>::value();
#pragma unroll
                for (int k = 0; k < Q; ++k) out[k] = solid ? M : out[k];
            }
        }
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int dx = X::dx(b), dy = X::dy(b);
            side[b * NPOS + my_pos] = V4<T>{out[kdir(dx, dy, -1)], out[kdir(dx, dy, 0)], out[kdir(dx, dy, 1)], T(0)};
        });
        static_for<0, ND>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            diag[j * NPOS + my_pos] = out[kdir(X::ddx(j), X::ddy(j), 0)];
        });
        if (hmode >= 0) store_halo_exports<Q, T>(side, diag, hplan, r_halo, a);
        if (p + 1 <= z1) prefetch(p + 1);
        __syncthreads();

        // gather this arrival's values by direction k
        T dn[Q], mid[Q], up_out[Q];  // c_z = -1 (for plane p-1), 0 (plane p), +1 (plane p+1)
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int dx = X::dx(b), dy = X::dy(b);
            const V4<T> v = side[b * NPOS + pos_of(tx - dx, ty - dy, PW)];
            dn[kdir(dx, dy, -1)] = v.x;
            mid[kdir(dx, dy, 0)] = v.y;
            up_out[kdir(dx, dy, 1)] = v.z;
        });
        static_for<0, ND>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            constexpr int dx = X::ddx(j), dy = X::ddy(j);
            mid[kdir(dx, dy, 0)] = diag[j * NPOS + pos_of(tx - dx, ty - dy, PW)];
        });
        dn[KZM] = out[KZM];
        up_out[KZP] = out[KZP];

        // plane p - 1: add its c_z = -1 links and finish it
        if (p - 1 >= z0) {
            const bool fluid = active && !(flag_prev & FLAG_SOLID);
            const bool wall = fluid && (flag_prev & FLAG_WALL_LINK);
            if (__any_sync(0xffffffffu, wall)) {
                static_for<1, Q>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    if constexpr (cvel(K, 2) == -1) {
                        if (Marker<T>::is(dn[K])) dn[K] = own_in[inv_dir(K)];
                    }
                });
            }
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                if constexpr (cvel(K, 2) == -1) acc.template add<K>(dn[K]);
            });
            if (fluid) {
                T dd, ux, uy, uz;
                node_finish<Q, T>(acc, dd, ux, uy, uz);
                const uint32_t i = (uint32_t)(p - 1) * nxy + out_xy;
                S::store(static_cast<st*>(a.post[0]), i, dd, a.scale[0]);
                S::store(static_cast<st*>(a.post[1]), i, ux, a.scale[1]);
                S::store(static_cast<st*>(a.post[2]), i, uy, a.scale[2]);
                S::store(static_cast<st*>(a.post[3]), i, uz, a.scale[3]);
            }
        }

        // plane p: the c_z = +1 links gathered last arrival and this arrival's c_z = 0 links
        if (p >= z0 && p < z1) {
            const bool fluid = active && !(cur.flag & FLAG_SOLID);
            const bool wall = fluid && (cur.flag & FLAG_WALL_LINK);
            if (__any_sync(0xffffffffu, wall)) {
                static_for<1, Q>([&](auto kc) {
                    constexpr int K = decltype(kc)::value;
                    if constexpr (cvel(K, 2) == 1) {
                        if (Marker<T>::is(up_in[K])) up_in[K] = out[inv_dir(K)];
                    } else if constexpr (cvel(K, 2) == 0) {
                        if (Marker<T>::is(mid[K])) mid[K] = out[inv_dir(K)];
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
        // carry to the next arrival
        static_for<1, Q>([&](auto kc) {
            constexpr int K = decltype(kc)::value;
            if constexpr (cvel(K, 2) == 1) {
                up_in[K] = up_out[K];
                own_in[K] = out[K];
            }
        });
        flag_prev = cur.flag;
    }
}

template <int Q, int ST> struct TileShape;
template <> struct TileShape<19, ST_F32> { static constexpr int TY = 8, MINB = 3; };
template <> struct TileShape<19, ST_F16S> { static constexpr int TY = 8, MINB = 3; };
template <> struct TileShape<19, ST_BF16S> { static constexpr int TY = 8, MINB = 3; };
template <> struct TileShape<19, ST_F64> { static constexpr int TY = 4, MINB = 1; };
template <> struct TileShape<27, ST_F32> { static constexpr int TY = 4, MINB = 4; };
template <> struct TileShape<27, ST_F16S> { static constexpr int TY = 4, MINB = 4; };
template <> struct TileShape<27, ST_BF16S> { static constexpr int TY = 4, MINB = 4; };
template <> struct TileShape<27, ST_F64> { static constexpr int TY = 4, MINB = 1; };

template <int Q, int ST>
cudaError_t launch_tiled_t(const StepArgs& a, cudaStream_t s)
{
    constexpr int TX = 32, TY = TileShape<Q, ST>::TY;
    using C = Cfg<Q, ST, TX, TY>;
    auto kern = tau1_tiled_kernel<Q, ST, TX, TY, TileShape<Q, ST>::MINB>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int ntx = (a.nx + TX - 1) / TX;
    const int nty = (a.ny + TY - 1) / TY;
    const int ntiles = ntx * nty;
    const int chunk = a.nz < 32 ? a.nz : 32;
    const int nchunks = (a.nz + chunk - 1) / chunk;
    const long long blocks = (long long)ntiles * nchunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, C::NT, C::SMEM, s>>>(a, ntx, ntiles, chunk);
    return cudaGetLastError();
}

}  // namespace

bool tau1_tiled_supported(int q, int storage, int64_t n)
{
    return (q == 19 || q == 27) && storage >= ST_F64 && storage <= ST_BF16S && n > 0 && n < ((int64_t)1 << 31);
}

cudaError_t launch_tau1_tiled(int q, int storage, const StepArgs& a, cudaStream_t s)
{
    switch (q * 10 + storage) {
    case 190 + ST_F64: return launch_tiled_t<19, ST_F64>(a, s);
    case 190 + ST_F32: return launch_tiled_t<19, ST_F32>(a, s);
    case 190 + ST_F16S: return launch_tiled_t<19, ST_F16S>(a, s);
    case 190 + ST_BF16S: return launch_tiled_t<19, ST_BF16S>(a, s);
    case 270 + ST_F64: return launch_tiled_t<27, ST_F64>(a, s);
    case 270 + ST_F32: return launch_tiled_t<27, ST_F32>(a, s);
    case 270 + ST_F16S: return launch_tiled_t<27, ST_F16S>(a, s);
    case 270 + ST_BF16S: return launch_tiled_t<27, ST_BF16S>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

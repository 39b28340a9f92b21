// Tau1 step for the D2Q9 lattice (one plane, nz = 1): the paper's 2D kernel
// (Section 3.1) and the lattice of its Poiseuille validation (Section 3.3).
//
// Two kernels with the same bits:
//   - tau1_simple2d: one thread per node, neighbours read from global memory
//     (the cross-check);
//   - tau1_march2d: each warp owns a strip of columns and marches along y. A
//     lane updates one column; the values a node sends along c_y = +1 wait in
//     registers for the next row, those along c_y = -1 complete the previous
//     row, and those along c_x = +-1 come from the neighbouring lane by warp
//     shuffle. Lanes 0 and 31 are halo columns: they are loaded and export,
//     and their own update is not stored (30 columns stored per warp), so no
//     value of a stored node comes from anywhere but registers and shuffles:
//     no shared memory, no block barrier.
//
// Per link (Eq. LBMTau1, Eq. feq with c_s^2 = 1/3): the source's equilibrium
// scaled by 1/w_k, A + p + p^2 H with p = c_k . 3 rho v (node_moments), or,
// for a wall source, the node's own value in direction inv(k) (Algorithm
// "Complete Tau1 ... halfway bounce-back") as fma(sigma, b, v). Links are
// accumulated per weight class in a fixed order (rest, then c_y = +1, 0, -1,
// each in k order); one reciprocal of rho at the end (Algorithm "Optimized
// Tau1 ... stores velocity").
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

// p = c_k . P (x term, then y term, so that p of inv(k) is exactly -p of k)
template <int K, typename T> __device__ __forceinline__ T dot2(T Px, T Py)
{
    constexpr int cx = c2(K, 0), cy = c2(K, 1);
    if constexpr (cx == 0) return cy > 0 ? Py : -Py;
    else {
        const T p = cx > 0 ? Px : -Px;
        if constexpr (cy == 0) return p;
        else return cy > 0 ? p + Py : p - Py;
    }
}

// Outgoing scaled equilibria of a node in all 9 directions (k / inv(k) share
// one fma chain, as in the 3D kernels); a solid node (drho NaN) exports 0 and
// has sigma = 1.
template <typename T>
__device__ __forceinline__ void exports2(T d, T ux, T uy, T gx, T gy, T (&out)[9], T& sigma)
{
    const bool solid = isnan(d);
    const NodeMoments<T> m0 = node_moments<T>(solid ? T(0) : d, ux, uy, T(0), gx, gy, T(0));
    const T keep = solid ? T(0) : T(1);
    sigma = solid ? T(1) : T(0);
    const T A = m0.A * keep, Px = m0.Px * keep, Py = m0.Py * keep;
    out[0] = A;
    static_for<0, 4>([&](auto ic) {
        constexpr int K = 1 + 2 * decltype(ic)::value;
        const T pk = dot2<K, T>(Px, Py);
        const T e = fma(pk * m0.H, pk, A);
        out[K] = e + pk;
        out[K + 1] = e - pk;
    });
}

// Per-class sums of one node; add() in the fixed link order.
template <typename T> struct Acc2 {
    T S[3], Jx[3], Jy[3];
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) S[c] = Jx[c] = Jy[c] = T(0);
    }
    template <int K> __device__ __forceinline__ void add(T f)
    {
        constexpr int c = class2(K);
        S[c] += f;
        if constexpr (c2(K, 0) > 0) Jx[c] += f;
        if constexpr (c2(K, 0) < 0) Jx[c] -= f;
        if constexpr (c2(K, 1) > 0) Jy[c] += f;
        if constexpr (c2(K, 1) < 0) Jy[c] -= f;
    }
    __device__ __forceinline__ void finish(T& d, T& ux, T& uy) const
    {
        T dd = T(w2(0)) * S[0];
        T jx = T(0), jy = T(0);
#pragma unroll
        for (int c = 1; c < 3; ++c) {
            dd = fma(T(w2(c)), S[c], dd);
            jx = fma(T(w2(c)), Jx[c], jx);
            jy = fma(T(w2(c)), Jy[c], jy);
        }
        const T r = recip(T(1) + dd);
        d = dd;
        ux = jx * r;
        uy = jy * r;
    }
};

// link order: c_y = +1 (k = 3, 5, 8), c_y = 0 (1, 2), c_y = -1 (4, 6, 7)
constexpr int ORDER_UP[3] = {3, 5, 8}, ORDER_MID[2] = {1, 2}, ORDER_DN[3] = {4, 6, 7};

__device__ __forceinline__ bool wrap2(int& c, int n, int periodic)
{
    if (c >= 0 && c < n) return true;
    if (!periodic) return false;
    c = c < 0 ? c + n : c - n;
    return c >= 0 && c < n;
}

template <int ST>
__global__ void __launch_bounds__(256) tau1_simple2d_kernel(StepArgs a)
{
    using S = Storage<ST>;
    using T = typename S::ctype;
    const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.nx || y >= a.ny) return;
    const Scales sc(a.dscale);
    const uint32_t i = (uint32_t)x + (uint32_t)a.nx * (uint32_t)y;
    T d0, ux0, uy0, uz0;
    S::load(a.pre, i, sc.inv, d0, ux0, uy0, uz0);
    if (isnan(d0)) return;
    const T gx = gcomp<T>(a, 0), gy = gcomp<T>(a, 1);
    T own[9], so;
    exports2<T>(d0, ux0, uy0, gx, gy, own, so);
    Acc2<T> acc;
    acc.clear();
    acc.template add<0>(own[0]);
    auto link = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        int sx = x - c2(K, 0), sy = y - c2(K, 1);
        T v = T(0), s = T(1);
        if (wrap2(sx, a.nx, a.periodic[0]) && wrap2(sy, a.ny, a.periodic[1])) {
            T d, ux, uy, uz, ex[9];
            S::load(a.pre, (uint32_t)sx + (uint32_t)a.nx * (uint32_t)sy, sc.inv, d, ux, uy, uz);
            exports2<T>(d, ux, uy, gx, gy, ex, s);
            v = ex[K];
        }
        acc.template add<K>(fma(s, own[inv2(K)], v));
    };
    static_for<0, 3>([&](auto j) { link(std::integral_constant<int, ORDER_UP[decltype(j)::value]>{}); });
    static_for<0, 2>([&](auto j) { link(std::integral_constant<int, ORDER_MID[decltype(j)::value]>{}); });
    static_for<0, 3>([&](auto j) { link(std::integral_constant<int, ORDER_DN[decltype(j)::value]>{}); });
    T d, ux, uy;
    acc.finish(d, ux, uy);
    step_store<ST>(a.post, i, d, ux, uy, T(0), sc.s, a.seed);
}

constexpr int M2_WARPS = 4;     // warps per block (independent)
constexpr int M2_COLS = 30;     // columns stored per warp

template <typename T> __device__ __forceinline__ T from_left(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T> __device__ __forceinline__ T from_right(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

template <int ST>
__global__ void __launch_bounds__(32 * M2_WARPS) tau1_march2d_kernel(StepArgs a, int ntx, int chunk, int nitems)
{
    using S = Storage<ST>;
    using T = typename S::ctype;
    const int item = blockIdx.x * M2_WARPS + (threadIdx.x >> 5);
    if (item >= nitems) return;  // whole warp
    const int lane = threadIdx.x & 31;
    const int tile = item % ntx, y0 = (item / ntx) * chunk;
    const int y1 = min(a.ny, y0 + chunk);
    const int xc = tile * M2_COLS - 1 + lane;  // this lane's column
    int xw = xc;
    const bool xok = wrap2(xw, a.nx, a.periodic[0]);
    const bool stores = lane >= 1 && lane <= M2_COLS && xc < a.nx;
    const Scales sc(a.dscale);
    const T gx = gcomp<T>(a, 0), gy = gcomp<T>(a, 1);

    auto load_row = [&](int p, T& d, T& ux, T& uy) {
        int yw = p;
        T uz;
        if (xok && wrap2(yw, a.ny, a.periodic[1])) {
            S::load(a.pre, (uint32_t)xw + (uint32_t)a.nx * (uint32_t)yw, sc.inv, d, ux, uy, uz);
        } else {
            d = T(NAN);
            ux = uy = T(0);
        }
    };

    // carried from row p - 1: its c_y = +1 values and sources' sigma for row p,
    // its own outgoing c_y = +1 values (bounce-back of its c_y = -1 links), its sums
    T up_v[3], up_s[3], own_up[3];
    Acc2<T> acc;
    acc.clear();
    bool fluid_prev = false;
#pragma unroll
    for (int j = 0; j < 3; ++j) up_v[j] = up_s[j] = own_up[j] = T(0);
    T nd, nux, nuy;
    load_row(y0 - 1, nd, nux, nuy);
    for (int p = y0 - 1; p <= y1; ++p) {
        const T d = nd, ux = nux, uy = nuy;
        if (p < y1) load_row(p + 1, nd, nux, nuy);  // next row in flight while this one computes
        T out[9], sig;
        exports2<T>(d, ux, uy, gx, gy, out, sig);
        const T sl = from_left(sig), sr = from_right(sig);
        // c_y = -1 values of row p complete row p - 1
        if (p > y0 - 1) {
            acc.template add<4>(fma(sig, own_up[0], out[4]));                    // (0,-1) from own column
            acc.template add<6>(fma(sr, own_up[1], from_right(out[6])));          // (-1,-1) from x + 1
            acc.template add<7>(fma(sl, own_up[2], from_left(out[7])));           // (+1,-1) from x - 1
            T dn, uxn, uyn;
            acc.finish(dn, uxn, uyn);
            if (stores && fluid_prev && p - 1 >= y0)
                step_store<ST>(a.post, (uint32_t)xc + (uint32_t)a.nx * (uint32_t)(p - 1), dn, uxn, uyn, T(0), sc.s,
                               a.seed);
        }
        if (p == y1) break;
        // row p: rest, the c_y = +1 values carried from row p - 1, then c_y = 0
        acc.clear();
        acc.template add<0>(out[0]);
        acc.template add<3>(fma(up_s[0], out[inv2(3)], up_v[0]));
        acc.template add<5>(fma(up_s[1], out[inv2(5)], up_v[1]));
        acc.template add<8>(fma(up_s[2], out[inv2(8)], up_v[2]));
        acc.template add<1>(fma(sl, out[inv2(1)], from_left(out[1])));
        acc.template add<2>(fma(sr, out[inv2(2)], from_right(out[2])));
        // c_y = +1 values of row p for row p + 1; own (., +1) values for its bounce-back
        up_v[0] = out[3];
        up_s[0] = sig;
        up_v[1] = from_left(out[5]);
        up_s[1] = sl;
        up_v[2] = from_right(out[8]);
        up_s[2] = sr;
        own_up[0] = out[inv2(4)];
        own_up[1] = out[inv2(6)];
        own_up[2] = out[inv2(7)];
        fluid_prev = sig == T(0);
    }
}

template <int ST> cudaError_t launch2(bool simple, const StepArgs& a, cudaStream_t s)
{
    if (simple) {
        const dim3 grid((unsigned)((a.nx + 31) / 32), (unsigned)((a.ny + 7) / 8));
        tau1_simple2d_kernel<ST><<<grid, 256, 0, s>>>(a);
    } else {
        const int ntx = (a.nx + M2_COLS - 1) / M2_COLS;
        // Rows per warp: long enough to amortise the two halo rows (about 64),
        // and chosen so that the warps fill a whole number of waves of the
        // warps the GPU holds at once (a last, partly filled wave leaves SMs
        // idle while the others finish). A node's result does not depend on it.
        auto kern = tau1_march2d_kernel<ST>;
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * M2_WARPS, 0);
        if (e != cudaSuccess) return e;
        const long long resident = (long long)sms * (per_sm > 0 ? per_sm : 1) * M2_WARPS;
        const long long cols = (long long)ntx;
        const long long at64 = cols * ((a.ny + 63) / 64);
        const long long waves = at64 / resident > 0 ? (at64 + resident / 2) / resident : 1;
        long long rows_per_col = waves * resident / cols;  // warps per column of tiles
        if (rows_per_col < 1) rows_per_col = 1;
        long long chunk_l = (a.ny + rows_per_col - 1) / rows_per_col;
        chunk_l = chunk_l < 8 ? 8 : (chunk_l > 128 ? 128 : chunk_l);
        const int chunk = (int)chunk_l;
        const long long items = cols * ((a.ny + chunk - 1) / chunk);
        if (items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        const unsigned blocks = (unsigned)((items + M2_WARPS - 1) / M2_WARPS);
        tau1_march2d_kernel<ST><<<blocks, 32 * M2_WARPS, 0, s>>>(a, ntx, chunk, (int)items);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tau1_2d(bool simple, int storage, const StepArgs& a, cudaStream_t s)
{
    if (a.nz != 1) return cudaErrorInvalidValue;
    switch (storage) {
    case ST_F64: return launch2<ST_F64>(simple, a, s);
    case ST_F32: return launch2<ST_F32>(simple, a, s);
    case ST_F16S: return launch2<ST_F16S>(simple, a, s);
    case ST_BF16S: return launch2<ST_BF16S>(simple, a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

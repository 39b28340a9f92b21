// Per-node arithmetic of the Tau1 update shared by the CUDA kernels.
//
// Eq. (feq) with c_s^2 = 1/3, written as the deviation from the rest weight
// and divided by the weight w_k:
//     (f_k^eq - w_k) / w_k = drho + rho (3 c.v + 4.5 (c.v)^2 - 1.5 v.v)
//                          = A + p + p^2 H,   p = c_k . P,
// with the per-node moments A = drho - 1.5 rho v.v, P = 3 rho v, H = 1/(2 rho)
// and v = u + g (velocity-shift body force). The weight is applied once per
// class of directions at the end of the node update.
#pragma once

#include "common.cuh"

namespace lbm {

template <typename T> struct NodeMoments {
    T A, Px, Py, Pz, H;
};

template <typename T>
__device__ __forceinline__ NodeMoments<T> node_moments(T drho, T ux, T uy, T uz, T gx, T gy, T gz)
{
    // Every fused multiply-add is written out, so that no kernel depends on
    // the compiler's contraction choices (the packed two-node kernels and the
    // scalar kernels then round identically).
    NodeMoments<T> m;
    const T rho = T(1) + drho;
    const T vx = ux + gx, vy = uy + gy, vz = uz + gz;
    const T vv = fma(vz, vz, fma(vy, vy, vx * vx));
    m.A = fma(T(-1.5) * rho, vv, drho);
    const T r3 = T(3) * rho;
    m.Px = r3 * vx;
    m.Py = r3 * vy;
    m.Pz = r3 * vz;
    m.H = T(0.5) * recip(rho);
    return m;
}

// p = c_k . P with compile-time velocity components (adds and subtractions in
// axis order x, y, z, so that p of inv(k) is exactly -p of k).
template <int K, typename T>
__device__ __forceinline__ T dir_dot(T Px, T Py, T Pz)
{
    constexpr int cx = cvel(K, 0), cy = cvel(K, 1), cz = cvel(K, 2);
    T p = T(0);
    bool any = false;
    if (cx != 0) { p = cx > 0 ? Px : -Px; any = true; }
    if (cy != 0) { p = any ? (cy > 0 ? p + Py : p - Py) : (cy > 0 ? Py : -Py); any = true; }
    if (cz != 0) { p = any ? (cz > 0 ? p + Pz : p - Pz) : (cz > 0 ? Pz : -Pz); any = true; }
    return p;
}

// (f_k^eq - w_k) / w_k from the source moments: A + p (1 + p H), evaluated as
// fma(p*H, p, A) + p. The value for inv(k) uses -p and is exact in sign.
template <typename T>
__device__ __forceinline__ T feq_scaled(T A, T H, T p)
{
    return fma(p * H, p, A) + p;
}

// Place of link K in the order in which the step kernels accumulate a node:
// the c_z = +1 links, then c_z = 0, then c_z = -1, each group in k order.
__host__ __device__ constexpr int acc_order(int k) { return (cvel(k, 2) == 1 ? 0 : (cvel(k, 2) == 0 ? 1 : 2)) * 32 + k; }

// True when link K is the first, in that order, to add to accumulator comp
// (0: S, 1..3: J_x..J_z) of its class. The sum then starts from that term
// instead of from zero: one addition fewer, and only the sign of an all-zero
// sum can differ.
template <int Q> __host__ __device__ constexpr bool first_link(int K, int comp)
{
    for (int k = 1; k < Q; ++k)
        if (dir_class(k) == dir_class(K) && (comp == 0 || cvel(k, comp - 1) != 0) && acc_order(k) < acc_order(K))
            return false;
    return true;
}

// Accumulators of one node: per direction class, the sum of the scaled
// equilibria and of c times them. add<Q, K> must be called in acc_order.
template <typename T, int NC> struct NodeAcc {
    T S[NC];
    T Jx[NC], Jy[NC], Jz[NC];
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int c = 0; c < NC; ++c) S[c] = Jx[c] = Jy[c] = Jz[c] = T(0);
    }
    template <int C, bool FIRST> __device__ static __forceinline__ void put(T& a, T f)
    {
        if constexpr (C > 0) {
            if constexpr (FIRST) a = f;
            else a += f;
        } else if constexpr (C < 0) {
            if constexpr (FIRST) a = -f;
            else a -= f;
        }
    }
    template <int Q, int K> __device__ __forceinline__ void add(T f)
    {
        constexpr int cls = dir_class(K);
        put<1, first_link<Q>(K, 0)>(S[cls], f);
        put<cvel(K, 0), first_link<Q>(K, 1)>(Jx[cls], f);
        put<cvel(K, 1), first_link<Q>(K, 2)>(Jy[cls], f);
        put<cvel(K, 2), first_link<Q>(K, 3)>(Jz[cls], f);
    }
};

// Final step of Algorithm "Optimized Tau1 ... stores velocity": apply the
// class weights, then one reciprocal of rho for the three velocity components.
template <int Q, typename T>
__device__ __forceinline__ void node_finish(const NodeAcc<T, Weights<Q>::NCLASS>& a, T& drho, T& ux, T& uy, T& uz)
{
    constexpr int NC = Weights<Q>::NCLASS;
    T d = T(Weights<Q>::w(0)) * a.S[0];
    T jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int c = 1; c < NC; ++c) {
        const T w = T(Weights<Q>::w(c));
        d = fma(w, a.S[c], d);
        jx = fma(w, a.Jx[c], jx);
        jy = fma(w, a.Jy[c], jy);
        jz = fma(w, a.Jz[c], jz);
    }
    const T r = recip(T(1) + d);
    drho = d;
    ux = jx * r;
    uy = jy * r;
    uz = jz * r;
}

}  // namespace lbm

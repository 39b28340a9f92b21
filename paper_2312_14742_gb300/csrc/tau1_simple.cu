// Tau1 step, one thread per node, neighbours read straight from global memory.
//
// The plain form of Algorithm "Tau1" (pull, AB layout) with the halfway
// bounce-back of Algorithm "Complete Tau1 ... halfway bounce-back": for each
// direction k the node gathers (drho, u) of x - c_k, forms the scaled
// equilibrium and accumulates it; a wall link takes the equilibrium of the
// node's own previous state in direction inv(k). It serves any box shape and
// every storage format, and is the cross-check of the tiled kernel.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

template <int Q, int ST>
__global__ void __launch_bounds__(256) tau1_simple_kernel(StepArgs a)
{
    using S = Storage<ST>;
    using T = typename S::ctype;
    using st = typename S::stype;
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (a.flags[i] & FLAG_SOLID) return;
    const int x = (int)(i % a.nx);
    const int y = (int)((i / a.nx) % a.ny);
    const int z = (int)(i / ((int64_t)a.nx * a.ny));
    const st* pre0 = static_cast<const st*>(a.pre[0]);
    const st* pre1 = static_cast<const st*>(a.pre[1]);
    const st* pre2 = static_cast<const st*>(a.pre[2]);
    const st* pre3 = static_cast<const st*>(a.pre[3]);
    const T gx = gcomp<T>(a, 0), gy = gcomp<T>(a, 1), gz = gcomp<T>(a, 2);

    const NodeMoments<T> own = node_moments<T>(S::load(pre0, i, a.inv_scale[0]), S::load(pre1, i, a.inv_scale[1]),
                                               S::load(pre2, i, a.inv_scale[2]), S::load(pre3, i, a.inv_scale[3]),
                                               gx, gy, gz);
    NodeAcc<T, Weights<Q>::NCLASS> acc;
    acc.clear();
    acc.S[0] = own.A;  // rest direction: p = 0

    // one link: the equilibrium arriving along c_K
    auto link = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        int sx = x - cvel(K, 0), sy = y - cvel(K, 1), sz = z - cvel(K, 2);
        bool wall = false;
        if (sx < 0 || sx >= a.nx) { if (a.periodic[0]) sx = sx < 0 ? sx + a.nx : sx - a.nx; else wall = true; }
        if (sy < 0 || sy >= a.ny) { if (a.periodic[1]) sy = sy < 0 ? sy + a.ny : sy - a.ny; else wall = true; }
        if (sz < 0 || sz >= a.nz) { if (a.periodic[2]) sz = sz < 0 ? sz + a.nz : sz - a.nz; else wall = true; }
        int64_t s = 0;
        if (!wall) {
            s = (int64_t)sx + (int64_t)a.nx * ((int64_t)sy + (int64_t)a.ny * sz);
            wall = (a.flags[s] & FLAG_SOLID) != 0;
        }
        T f;
        if (wall) {
            // reflected population: own state in direction inv(k), p(inv k) = -p(k)
            const T p = -dir_dot<K, T>(own.Px, own.Py, own.Pz);
            f = feq_scaled(own.A, own.H, p);
        } else {
            const NodeMoments<T> m = node_moments<T>(S::load(pre0, s, a.inv_scale[0]), S::load(pre1, s, a.inv_scale[1]),
                                                     S::load(pre2, s, a.inv_scale[2]), S::load(pre3, s, a.inv_scale[3]),
                                                     gx, gy, gz);
            f = feq_scaled(m.A, m.H, dir_dot<K, T>(m.Px, m.Py, m.Pz));
        }
        acc.template add<K>(f);
    };
    // Accumulation order: links with c_z = +1, then 0, then -1, each in k
    // order (the order in which the z-marching kernels receive them), so all
    // kernels give the same bits.
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 1) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 0) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == -1) link(kc); });

    T d, ux, uy, uz;
    node_finish<Q, T>(acc, d, ux, uy, uz);
    S::store(static_cast<st*>(a.post[0]), i, d, a.scale[0]);
    S::store(static_cast<st*>(a.post[1]), i, ux, a.scale[1]);
    S::store(static_cast<st*>(a.post[2]), i, uy, a.scale[2]);
    S::store(static_cast<st*>(a.post[3]), i, uz, a.scale[3]);
}

template <int Q, int ST>
static cudaError_t launch_simple_t(const StepArgs& a, cudaStream_t s)
{
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    const int64_t blocks = (n + 255) / 256;
    tau1_simple_kernel<Q, ST><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tau1_simple(int q, int storage, const StepArgs& a, cudaStream_t s)
{
    switch (q * 10 + storage) {
    case 190 + ST_F64: return launch_simple_t<19, ST_F64>(a, s);
    case 190 + ST_F32: return launch_simple_t<19, ST_F32>(a, s);
    case 190 + ST_F16S: return launch_simple_t<19, ST_F16S>(a, s);
    case 190 + ST_BF16S: return launch_simple_t<19, ST_BF16S>(a, s);
    case 270 + ST_F64: return launch_simple_t<27, ST_F64>(a, s);
    case 270 + ST_F32: return launch_simple_t<27, ST_F32>(a, s);
    case 270 + ST_F16S: return launch_simple_t<27, ST_F16S>(a, s);
    case 270 + ST_BF16S: return launch_simple_t<27, ST_BF16S>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

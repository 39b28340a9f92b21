// Tau1 step, one thread per node, neighbours read straight from global memory.
//
// The plain form of Algorithm "Tau1" (pull, AB layout) with the halfway
// bounce-back of Algorithm "Complete Tau1 ... halfway bounce-back": for each
// direction k the node gathers (drho, u) of x - c_k, forms the scaled
// equilibrium and accumulates it; a wall link takes the equilibrium of the
// node's own previous state in direction inv(k). It serves any box shape and
// every storage format and is the cross-check of the tiled kernel: it
// evaluates each link with the same operations in the same order (walls as
// fma(sigma, b, v) with sigma = 1 for a wall, 0 otherwise; links in the order
// c_z = +1, 0, -1, each in k order), so both kernels give the same bits.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

template <int Q, int ST>
__global__ void __launch_bounds__(256) tau1_simple_kernel(StepArgs a)
{
    using S = Storage<ST>;
    using T = typename S::ctype;
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Scales sc(a.dscale);
    T d0, ux0, uy0, uz0;
    S::load(a.pre, (uint32_t)i, sc.inv, d0, ux0, uy0, uz0);
    if (isnan(d0)) return;  // solid node
    const int x = (int)(i % a.nx);
    const int y = (int)((i / a.nx) % a.ny);
    const int z = (int)(i / ((int64_t)a.nx * a.ny));
    const T gx = gcomp<T>(a, 0), gy = gcomp<T>(a, 1), gz = gcomp<T>(a, 2);

    const NodeMoments<T> own = node_moments<T>(d0, ux0, uy0, uz0, gx, gy, gz);
    NodeAcc<T, Weights<Q>::NCLASS> acc;
    acc.S[0] = own.A;  // rest direction: p = 0

    // one link: the equilibrium arriving along c_K, or the reflected one
    auto link = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        int sx = x - cvel(K, 0), sy = y - cvel(K, 1), sz = z - cvel(K, 2);
        bool inside = true;
        if (sx < 0 || sx >= a.nx) { if (a.periodic[0]) sx = sx < 0 ? sx + a.nx : sx - a.nx; else inside = false; }
        if (sy < 0 || sy >= a.ny) { if (a.periodic[1]) sy = sy < 0 ? sy + a.ny : sy - a.ny; else inside = false; }
        if (sz < 0 || sz >= a.nz) { if (a.periodic[2]) sz = sz < 0 ? sz + a.nz : sz - a.nz; else inside = false; }
        T d = T(0), ux = T(0), uy = T(0), uz = T(0);
        bool solid = true;
        if (inside) {
            const int64_t s = (int64_t)sx + (int64_t)a.nx * ((int64_t)sy + (int64_t)a.ny * sz);
            S::load(a.pre, (uint32_t)s, sc.inv, d, ux, uy, uz);
            solid = isnan(d);
            if (solid) d = T(0);
        }
        // source value; a wall source contributes 0 (its moments are zeroed)
        NodeMoments<T> m = node_moments<T>(d, ux, uy, uz, gx, gy, gz);
        const T keep = solid ? T(0) : T(1);
        m.A = m.A * keep;
        m.Px = m.Px * keep;
        m.Py = m.Py * keep;
        m.Pz = m.Pz * keep;
        const T v = feq_scaled(m.A, m.H, dir_dot<K, T>(m.Px, m.Py, m.Pz));
        // reflected population: own state in direction inv(k), p(inv k) = -p(k)
        const T b = feq_scaled(own.A, own.H, -dir_dot<K, T>(own.Px, own.Py, own.Pz));
        acc.template add<Q, K>(fma(solid ? T(1) : T(0), b, v));
    };
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 1) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == 0) link(kc); });
    static_for<1, Q>([&](auto kc) { if constexpr (cvel(decltype(kc)::value, 2) == -1) link(kc); });

    T d, ux, uy, uz;
    node_finish<Q, T>(acc, d, ux, uy, uz);
    step_store<ST>(a.post, (uint32_t)i, d, ux, uy, uz, sc.s, a.seed);
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

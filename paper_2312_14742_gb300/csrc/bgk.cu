// Standard BGK lattice Boltzmann at tau = 1 with stored populations: the
// comparison kernel for Tau1 (Algorithm "Standard LBM", pull scheme, AB
// layout; Eq. LBGK with tau = 1 so the post-collision population is the
// equilibrium).
//
// Populations are stored per direction (f[k][node], one array per k) as
// deviations h_k = f_k - w_k, which is the same quantity with the rest
// weight taken out, so FP32 keeps the small part. The arrays hold
// post-collision populations of the previous step. One step: gather
// h_k(x - c_k) (a wall source: h_{inv k}(x), halfway bounce-back), moments
// drho = sum h, j = sum c h, u = j / rho, equilibrium at v = u + g
// (velocity-shift force, the same as the Tau1 kernels), store the q
// equilibria. Traffic: q values read and q written per fluid node, the 2 q s
// bytes of Table "tab_complexity". Solid nodes hold NaN populations.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

template <typename T> struct BgkArgs {
    int nx, ny, nz;
    int periodic[3];
    T g[3];
    const T* fin;  // [q][n]
    T* fout;       // [q][n]
    void* state;   // moments kernel output (records), or null
};

template <int Q, typename T>
__device__ __forceinline__ void heq_all(T drho, T ux, T uy, T uz, T gx, T gy, T gz, T (&h)[Q])
{
    const NodeMoments<T> m = node_moments<T>(drho, ux, uy, uz, gx, gy, gz);
    h[0] = T(Weights<Q>::w(0)) * m.A;
    static_for<1, Q>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        h[K] = T(Weights<Q>::w(dir_class(K))) * feq_scaled(m.A, m.H, dir_dot<K, T>(m.Px, m.Py, m.Pz));
    });
}

// Gathered populations of node i (pull with halfway bounce-back) and their moments.
template <int Q, typename T>
__device__ __forceinline__ bool gather(const BgkArgs<T>& a, int64_t i, int64_t n, T (&hp)[Q], T& drho, T& ux, T& uy,
                                       T& uz)
{
    if (isnan(a.fin[i])) return false;  // solid node
    const int x = (int)(i % a.nx), y = (int)((i / a.nx) % a.ny), z = (int)(i / ((int64_t)a.nx * a.ny));
    static_for<0, Q>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        int sx = x - cvel(K, 0), sy = y - cvel(K, 1), sz = z - cvel(K, 2);
        bool inside = true;
        if (sx < 0 || sx >= a.nx) { if (a.periodic[0]) sx = sx < 0 ? sx + a.nx : sx - a.nx; else inside = false; }
        if (sy < 0 || sy >= a.ny) { if (a.periodic[1]) sy = sy < 0 ? sy + a.ny : sy - a.ny; else inside = false; }
        if (sz < 0 || sz >= a.nz) { if (a.periodic[2]) sz = sz < 0 ? sz + a.nz : sz - a.nz; else inside = false; }
        T v = T(NAN);
        if (inside) v = a.fin[(int64_t)K * n + (int64_t)sx + (int64_t)a.nx * ((int64_t)sy + (int64_t)a.ny * sz)];
        if (isnan(v)) v = a.fin[(int64_t)inv_dir(K) * n + i];
        hp[K] = v;
    });
    T d = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        d = d + hp[k];
        if (cvel(k, 0) > 0) jx = jx + hp[k]; else if (cvel(k, 0) < 0) jx = jx - hp[k];
        if (cvel(k, 1) > 0) jy = jy + hp[k]; else if (cvel(k, 1) < 0) jy = jy - hp[k];
        if (cvel(k, 2) > 0) jz = jz + hp[k]; else if (cvel(k, 2) < 0) jz = jz - hp[k];
    }
    const T r = T(1) / (T(1) + d);
    drho = d;
    ux = jx * r;
    uy = jy * r;
    uz = jz * r;
    return true;
}

template <int Q, typename T>
__global__ void __launch_bounds__(256) bgk_step_kernel(BgkArgs<T> a)
{
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T hp[Q], d, ux, uy, uz;
    if (!gather<Q, T>(a, i, n, hp, d, ux, uy, uz)) return;
    T h[Q];
    heq_all<Q, T>(d, ux, uy, uz, a.g[0], a.g[1], a.g[2], h);
#pragma unroll
    for (int k = 0; k < Q; ++k) a.fout[(int64_t)k * n + i] = h[k];
}

// Moments of the populations each node would gather now: the state that
// Tau1 reports after the same number of steps.
template <int Q, typename T>
__global__ void __launch_bounds__(256) bgk_moments_kernel(BgkArgs<T> a)
{
    using S = Storage<sizeof(T) == 8 ? ST_F64 : ST_F32>;
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T hp[Q], d, ux, uy, uz;
    if (!gather<Q, T>(a, i, n, hp, d, ux, uy, uz)) {
        S::store(a.state, (uint32_t)i, T(NAN), T(0), T(0), T(0), nullptr);
        return;
    }
    S::store(a.state, (uint32_t)i, d, ux, uy, uz, nullptr);
}

// Post-collision populations of a state (records; NaN drho = solid).
template <int Q, typename T>
__global__ void __launch_bounds__(256) bgk_init_kernel(BgkArgs<T> a)
{
    using S = Storage<sizeof(T) == 8 ? ST_F64 : ST_F32>;
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T d, ux, uy, uz;
        S::load(a.state, (uint32_t)i, nullptr, d, ux, uy, uz);
        T h[Q];
        if (isnan(d)) {
#pragma unroll
            for (int k = 0; k < Q; ++k) h[k] = T(NAN);
        } else {
            heq_all<Q, T>(d, ux, uy, uz, a.g[0], a.g[1], a.g[2], h);
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) a.fout[(int64_t)k * n + i] = h[k];
    }
}

template <typename T> BgkArgs<T> make_args(const StepArgs& s, const void* fin, void* fout, void* state)
{
    BgkArgs<T> a;
    a.nx = s.nx;
    a.ny = s.ny;
    a.nz = s.nz;
    for (int d = 0; d < 3; ++d) {
        a.periodic[d] = s.periodic[d];
        a.g[d] = sizeof(T) == 8 ? (T)s.g[d] : (T)s.gf[d];
    }
    a.fin = static_cast<const T*>(fin);
    a.fout = static_cast<T*>(fout);
    a.state = state;
    return a;
}

template <int Q, typename T> cudaError_t run(int what, const StepArgs& s, const void* fin, void* fout, void* state,
                                             cudaStream_t st)
{
    const int64_t n = (int64_t)s.nx * s.ny * s.nz;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const BgkArgs<T> a = make_args<T>(s, fin, fout, state);
    if (what == 0) bgk_step_kernel<Q, T><<<blocks, 256, 0, st>>>(a);
    else if (what == 1) bgk_moments_kernel<Q, T><<<blocks, 256, 0, st>>>(a);
    else bgk_init_kernel<Q, T><<<blocks < 152 * 64 ? blocks : 152 * 64, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t dispatch(int what, int q, int storage, const StepArgs& s, const void* fin, void* fout, void* state,
                     cudaStream_t st)
{
    if (q == 19 && storage == ST_F32) return run<19, float>(what, s, fin, fout, state, st);
    if (q == 19 && storage == ST_F64) return run<19, double>(what, s, fin, fout, state, st);
    if (q == 27 && storage == ST_F32) return run<27, float>(what, s, fin, fout, state, st);
    if (q == 27 && storage == ST_F64) return run<27, double>(what, s, fin, fout, state, st);
    return cudaErrorInvalidValue;
}

}  // namespace

bool bgk_supported(int q, int storage) { return (q == 19 || q == 27) && (storage == ST_F32 || storage == ST_F64); }

cudaError_t launch_bgk_step(int q, int storage, const StepArgs& a, const void* fin, void* fout, cudaStream_t s)
{
    return dispatch(0, q, storage, a, fin, fout, nullptr, s);
}

cudaError_t launch_bgk_moments(int q, int storage, const StepArgs& a, const void* fin, void* state, cudaStream_t s)
{
    return dispatch(1, q, storage, a, fin, nullptr, state, s);
}

cudaError_t launch_bgk_init(int q, int storage, const StepArgs& a, const void* state, void* fout, cudaStream_t s)
{
    return dispatch(2, q, storage, a, nullptr, fout, const_cast<void*>(state), s);
}

}  // namespace lbm

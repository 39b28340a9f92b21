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
// bytes of Table "tab_complexity", plus one 4-byte word of wall links.
//
// The wall links of every node are a bit mask built once from the geometry
// (bit k: the source x - c_k is solid or beyond a non-periodic face; bit 31:
// the node itself is solid), so each direction is one load from either the
// neighbour or the node's own opposite population, with no second dependent
// read. Threads are laid out as a 3D grid (32 x 8 nodes of a plane per
// block, one plane per grid z), so no thread divides to find its position.
// Solid nodes hold NaN populations and are never written.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

constexpr uint32_t BGK_SOLID = 1u << 31;
constexpr int BX = 32, BY = 8;

template <typename T> struct BgkArgs {
    int nx, ny, nz;
    int periodic[3];
    T g[3];
    const T* fin;          // [q][n]
    T* fout;               // [q][n]
    void* state;           // moments kernel output (records), or null
    const uint32_t* mask;  // wall links per node
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

__device__ __forceinline__ int wrap1(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// Gathered populations of node (x, y, z) (pull with halfway bounce-back) and
// their moments; false for a solid node.
template <int Q, typename T>
__device__ __forceinline__ bool gather(const BgkArgs<T>& a, int x, int y, int z, int64_t& i, T (&hp)[Q], T& drho,
                                       T& ux, T& uy, T& uz)
{
    const int64_t nxy = (int64_t)a.nx * a.ny, n = nxy * a.nz;
    i = (int64_t)x + (int64_t)a.nx * y + nxy * z;
    const uint32_t m = a.mask[i];
    if (m & BGK_SOLID) return false;
    // coordinate of x - c for c = -1, 0, +1 (wrapped; a source beyond a
    // non-periodic face is a wall by the mask and its index is not used)
    const int64_t X[3] = {wrap1(x + 1, a.nx), x, wrap1(x - 1, a.nx)};
    const int64_t Y[3] = {(int64_t)a.nx * wrap1(y + 1, a.ny), (int64_t)a.nx * y, (int64_t)a.nx * wrap1(y - 1, a.ny)};
    const int64_t Z[3] = {nxy * wrap1(z + 1, a.nz), nxy * z, nxy * wrap1(z - 1, a.nz)};
    static_for<0, Q>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        const int64_t j = X[cvel(K, 0) + 1] + Y[cvel(K, 1) + 1] + Z[cvel(K, 2) + 1];
        const T* p = ((m >> K) & 1u) ? a.fin + (int64_t)inv_dir(K) * n + i : a.fin + (int64_t)K * n + j;
        hp[K] = __ldg(p);
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
__global__ void __launch_bounds__(BX * BY) bgk_step_kernel(BgkArgs<T> a)
{
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    for (int z = blockIdx.z; z < a.nz; z += gridDim.z) {
        T hp[Q], d, ux, uy, uz;
        int64_t i;
        if (!gather<Q, T>(a, x, y, z, i, hp, d, ux, uy, uz)) continue;
        T h[Q];
        heq_all<Q, T>(d, ux, uy, uz, a.g[0], a.g[1], a.g[2], h);
#pragma unroll
        for (int k = 0; k < Q; ++k) a.fout[(int64_t)k * n + i] = h[k];
    }
}

// Moments of the populations each node would gather now: the state that
// Tau1 reports after the same number of steps.
template <int Q, typename T>
__global__ void __launch_bounds__(BX * BY) bgk_moments_kernel(BgkArgs<T> a)
{
    using S = Storage<sizeof(T) == 8 ? ST_F64 : ST_F32>;
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    for (int z = blockIdx.z; z < a.nz; z += gridDim.z) {
        T hp[Q], d, ux, uy, uz;
        int64_t i;
        if (!gather<Q, T>(a, x, y, z, i, hp, d, ux, uy, uz)) {
            S::store(a.state, (uint32_t)i, T(NAN), T(0), T(0), T(0), nullptr);
            continue;
        }
        S::store(a.state, (uint32_t)i, d, ux, uy, uz, nullptr);
    }
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

// Wall links of every node from the node flags (see the top of the file).
template <int Q>
__global__ void __launch_bounds__(BX * BY) bgk_mask_kernel(int nx, int ny, int nz, int px, int py, int pz,
                                                           const uint8_t* flags, uint32_t* mask)
{
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int64_t nxy = (int64_t)nx * ny;
    for (int z = blockIdx.z; z < nz; z += gridDim.z) {
        const int64_t i = (int64_t)x + (int64_t)nx * y + nxy * z;
        uint32_t m = 0;
        if (flags[i] & FLAG_SOLID) {
            m = BGK_SOLID;
        } else {
            static_for<1, Q>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                int sx = x - cvel(K, 0), sy = y - cvel(K, 1), sz = z - cvel(K, 2);
                bool wall = false;
                if (sx < 0 || sx >= nx) { if (px) sx = wrap1(sx, nx); else wall = true; }
                if (sy < 0 || sy >= ny) { if (py) sy = wrap1(sy, ny); else wall = true; }
                if (sz < 0 || sz >= nz) { if (pz) sz = wrap1(sz, nz); else wall = true; }
                if (!wall) wall = (flags[(int64_t)sx + (int64_t)nx * sy + nxy * sz] & FLAG_SOLID) != 0;
                if (wall) m |= 1u << K;
            });
        }
        mask[i] = m;
    }
}

template <typename T>
BgkArgs<T> make_args(const StepArgs& s, const void* fin, void* fout, void* state, const uint32_t* mask)
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
    a.mask = mask;
    return a;
}

dim3 grid3(int nx, int ny, int nz)
{
    return dim3((unsigned)((nx + BX - 1) / BX), (unsigned)((ny + BY - 1) / BY), (unsigned)(nz < 65535 ? nz : 65535));
}

template <int Q, typename T>
cudaError_t run(int what, const StepArgs& s, const void* fin, void* fout, void* state, const uint32_t* mask,
                cudaStream_t st)
{
    const int64_t n = (int64_t)s.nx * s.ny * s.nz;
    const BgkArgs<T> a = make_args<T>(s, fin, fout, state, mask);
    const dim3 block(BX, BY);
    if (what == 0) bgk_step_kernel<Q, T><<<grid3(s.nx, s.ny, s.nz), block, 0, st>>>(a);
    else if (what == 1) bgk_moments_kernel<Q, T><<<grid3(s.nx, s.ny, s.nz), block, 0, st>>>(a);
    else {
        const int64_t blocks = (n + 255) / 256;
        bgk_init_kernel<Q, T><<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t dispatch(int what, int q, int storage, const StepArgs& s, const void* fin, void* fout, void* state,
                     const uint32_t* mask, cudaStream_t st)
{
    if (q == 19 && storage == ST_F32) return run<19, float>(what, s, fin, fout, state, mask, st);
    if (q == 19 && storage == ST_F64) return run<19, double>(what, s, fin, fout, state, mask, st);
    if (q == 27 && storage == ST_F32) return run<27, float>(what, s, fin, fout, state, mask, st);
    if (q == 27 && storage == ST_F64) return run<27, double>(what, s, fin, fout, state, mask, st);
    return cudaErrorInvalidValue;
}

}  // namespace

bool bgk_supported(int q, int storage) { return (q == 19 || q == 27) && (storage == ST_F32 || storage == ST_F64); }

cudaError_t launch_bgk_mask(int q, const StepArgs& a, const uint8_t* flags, uint32_t* mask, cudaStream_t s)
{
    const dim3 grid = grid3(a.nx, a.ny, a.nz), block(BX, BY);
    if (q == 19) bgk_mask_kernel<19><<<grid, block, 0, s>>>(a.nx, a.ny, a.nz, a.periodic[0], a.periodic[1],
                                                            a.periodic[2], flags, mask);
    else if (q == 27) bgk_mask_kernel<27><<<grid, block, 0, s>>>(a.nx, a.ny, a.nz, a.periodic[0], a.periodic[1],
                                                                 a.periodic[2], flags, mask);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_bgk_step(int q, int storage, const StepArgs& a, const void* fin, void* fout, const uint32_t* mask,
                            cudaStream_t s)
{
    return dispatch(0, q, storage, a, fin, fout, nullptr, mask, s);
}

cudaError_t launch_bgk_moments(int q, int storage, const StepArgs& a, const void* fin, void* state,
                               const uint32_t* mask, cudaStream_t s)
{
    return dispatch(1, q, storage, a, fin, nullptr, state, mask, s);
}

cudaError_t launch_bgk_init(int q, int storage, const StepArgs& a, const void* state, void* fout, cudaStream_t s)
{
    return dispatch(2, q, storage, a, nullptr, fout, const_cast<void*>(state), nullptr, s);
}

}  // namespace lbm

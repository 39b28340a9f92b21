// Per-field power-of-two scales of the 16-bit storage formats, kept on the
// device and re-chosen there, so that stepping never waits for the host.
//
// FP16 keeps 11 significant bits between 2^-14 and 65504. Each field f of
// the state is stored as value * S_f with S_f = 2^e_f. The headroom rule:
// with m_f the largest |value| of field f over fluid nodes, the reference
// magnitude is r_f = max(m_f, max_f' m_f' / 16, 64 |g|_max), and S_f is
// chosen so that r_f * S_f = 2^12 (2^4 below the largest finite FP16);
// it is re-chosen when m_f * S_f rises above 2^13 or r_f * S_f falls below
// 2^9. The two floors keep a field that is still near zero (drho and the
// transverse velocities of a driven flow start at rounding level) from
// taking a scale so large that its growth over the 64 steps between checks
// overflows: a field may grow 16x in that time, from the larger of the
// other fields' size and what the body force adds in 64 steps. Below the
// floor FP16 still resolves values down to r_f * 2^-36 absolutely.
// Re-scaling multiplies the stored values by a power of two, which is exact
// away from the subnormal range. BF16 has the FP32 exponent range and keeps
// S_f = 1.
//
// Device layout of the scales: float[8] = {S_0..S_3, 1/S_0..1/S_3}.
#include <cmath>

#include "kernels.h"

namespace lbm {

namespace {

constexpr int AB = 256;  // threads per absmax block
constexpr double scale_force_steps = 64;  // the floor 64 |g|_max

template <int ST>
__global__ void __launch_bounds__(AB) absmax_state_kernel(int64_t n, const void* state, const uint8_t* __restrict__ flags,
                                                          const float* __restrict__ dscale, float* __restrict__ partial)
{
    using S = Storage<ST>;
    __shared__ float sm[4][AB];
    float inv[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) inv[f] = dscale[4 + f];
    float m[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * AB + threadIdx.x; i < n; i += (int64_t)gridDim.x * AB) {
        if (flags && (flags[i] & FLAG_SOLID)) continue;
        float v[4];
        S::load(state, (uint32_t)i, inv, v[0], v[1], v[2], v[3]);
#pragma unroll
        for (int f = 0; f < 4; ++f) m[f] = fmaxf(m[f], fabsf(v[f]));
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) sm[f][threadIdx.x] = m[f];
    __syncthreads();
    for (int w = AB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int f = 0; f < 4; ++f) sm[f][threadIdx.x] = fmaxf(sm[f][threadIdx.x], sm[f][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[blockIdx.x * 4 + threadIdx.x] = sm[threadIdx.x][0];
}

// One thread per field: new scale from the maxima; ratio[f] = S_new / S_old.
__global__ void decide_kernel(int blocks, const float* __restrict__ partial, float* dscale, float* ratio, int fp16,
                              float gfloor)
{
    const int f = threadIdx.x;
    if (f >= 4) return;
    float m[4] = {0.f, 0.f, 0.f, 0.f};
    for (int b = 0; b < blocks; ++b)
#pragma unroll
        for (int k = 0; k < 4; ++k) m[k] = fmaxf(m[k], partial[b * 4 + k]);
    const float mall = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
    const float ref = fmaxf(fmaxf(m[f], 0.0625f * mall), gfloor);
    const float s_old = dscale[f];
    float s_new = s_old;
    if (fp16 && ref > 0.f && isfinite(mall)) {
        if (m[f] * s_old > 8192.f || ref * s_old < 512.f) {
            int e;
            frexpf(ref, &e);  // ref = mant * 2^e, mant in [0.5, 1)
            e = 12 - e;
            e = e > 100 ? 100 : (e < -100 ? -100 : e);
            s_new = ldexpf(1.f, e);
        }
    }
    ratio[f] = s_new / s_old;
    dscale[f] = s_new;
    dscale[4 + f] = 1.f / s_new;
}

template <int ST>
__global__ void __launch_bounds__(AB) apply_kernel(int64_t n, void* state, const float* __restrict__ ratio)
{
    using S = Storage<ST>;
    const float r[4] = {ratio[0], ratio[1], ratio[2], ratio[3]};
    if (r[0] == 1.f && r[1] == 1.f && r[2] == 1.f && r[3] == 1.f) return;
    const float one[4] = {1.f, 1.f, 1.f, 1.f};
    for (int64_t i = (int64_t)blockIdx.x * AB + threadIdx.x; i < n; i += (int64_t)gridDim.x * AB) {
        float v[4];
        S::load(state, (uint32_t)i, one, v[0], v[1], v[2], v[3]);  // stored units
        S::store(state, (uint32_t)i, v[0], v[1], v[2], v[3], r);   // times the ratio (NaN stays NaN)
    }
}

int absmax_blocks(int64_t n)
{
    int64_t b = (n + AB * 16 - 1) / (AB * 16);
    return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

}  // namespace

// partial: absmax_blocks(n) * 4 floats; ratio: 4 floats (device).
cudaError_t launch_rescale(int storage, int64_t n, void* state, const uint8_t* flags, float* dscale, float* partial,
                           float* ratio, double gmax, cudaStream_t s)
{
    if (storage != ST_F16S && storage != ST_BF16S) return cudaSuccess;
    const int blocks = absmax_blocks(n);
    if (storage == ST_F16S) absmax_state_kernel<ST_F16S><<<blocks, AB, 0, s>>>(n, state, flags, dscale, partial);
    else absmax_state_kernel<ST_BF16S><<<blocks, AB, 0, s>>>(n, state, flags, dscale, partial);
    decide_kernel<<<1, 32, 0, s>>>(blocks, partial, dscale, ratio, storage == ST_F16S ? 1 : 0,
                                   (float)(scale_force_steps * gmax));
    if (storage == ST_F16S) apply_kernel<ST_F16S><<<blocks, AB, 0, s>>>(n, state, ratio);
    else apply_kernel<ST_BF16S><<<blocks, AB, 0, s>>>(n, state, ratio);
    return cudaGetLastError();
}

int rescale_scratch_floats(int64_t n) { return absmax_blocks(n) * 4 + 4; }

// Initial scales from the fields' maxima m[4] by the headroom rule (FP16;
// 1 for other formats, and for fields whose reference magnitude is 0).
void initial_scales(int storage, const double m[4], double gmax, float scale[4])
{
    double mall = 0;
    for (int f = 0; f < 4; ++f)
        if (std::isfinite(m[f])) mall = std::fmax(mall, m[f]);
    for (int f = 0; f < 4; ++f) {
        scale[f] = 1.0f;
        const double mf = std::isfinite(m[f]) ? m[f] : 0.0;
        const double ref = std::fmax(std::fmax(mf, mall / 16), scale_force_steps * gmax);
        if (storage != ST_F16S || !(ref > 0.0)) continue;
        int e;
        std::frexp(ref, &e);
        e = 12 - e;
        e = e > 100 ? 100 : (e < -100 ? -100 : e);
        scale[f] = std::ldexp(1.0f, e);
    }
}

}  // namespace lbm

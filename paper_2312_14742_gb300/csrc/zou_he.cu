// Constant-density (pressure) faces of Zou and He for the Tau1 step.
//
// The paper drives its 2D validation channel by a density rho_in at the
// inlet and rho_out at the outlet (Section 3.3). A fluid node on such a face
// of a non-periodic axis keeps its density; the populations that would enter
// from outside (c along the axis pointing into the box) are unknown. Zou and
// He set them so that the node's moments are (rho_b, u) with u along the
// axis, zero across it, and
//     rho_b (1 - s u) = sum_{c_a = 0} f + 2 sum_{c_a = -s} f,
// s = +1 on the face at coordinate 0, -1 on the face at n - 1. At tau = 1 the
// node's new state is exactly those moments, so Tau1 needs only the sums of
// the known populations: with f = w + h (h the deviation from the weight),
//     u = s (rho_b - 1 - H0 - 2 Hout) / rho_b.
// The known populations arrive as in the interior: the equilibrium of a fluid
// source x - c_k, or the halfway bounce-back value of a wall link.
//
// The step kernel updates the face nodes like any other (the faces of a
// non-periodic axis are walls to it); this kernel runs after it on the same
// stream, reads the same pre state, and overwrites the face nodes of the post
// state. One thread per face node. The face arithmetic is FP64 for every
// storage format: u is the difference of two sums of about rho_b - 1 each,
// and the faces are a small share of the nodes.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

template <int Q, int ST>
__global__ void __launch_bounds__(256) zou_he_kernel(StepArgs a, int axis, double rho_lo, double rho_hi)
{
    using S = Storage<ST>;
    using C = typename S::ctype;  // stored values
    using T = double;             // face arithmetic
    using LT = Lat<Q>;
    const int n[3] = {a.nx, a.ny, a.nz};
    const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;  // in-face axes
    const int64_t face = (int64_t)n[ua] * n[va];
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * face) return;
    const int side = t >= face ? 1 : 0;
    if (side && n[axis] == 1) return;  // one plane: the low face only
    t -= side * face;
    int pos[3];
    pos[axis] = side ? n[axis] - 1 : 0;
    pos[ua] = (int)(t % n[ua]);
    pos[va] = (int)(t / n[ua]);
    const uint32_t i = (uint32_t)pos[0] + (uint32_t)a.nx * ((uint32_t)pos[1] + (uint32_t)a.ny * (uint32_t)pos[2]);
    const Scales sc(a.dscale);
    C c0, c1, c2v, c3;
    S::load(a.pre, i, sc.inv, c0, c1, c2v, c3);
    if (isnan(c0)) return;  // solid face node
    const T d0 = c0, ux0 = c1, uy0 = c2v, uz0 = c3;
    // the step kernels evaluate g in the compute precision of the format
    const T gx = (T)gcomp<C>(a, 0), gy = (T)gcomp<C>(a, 1), gz = (T)gcomp<C>(a, 2);
    const NodeMoments<T> own = node_moments<T>(d0, ux0, uy0, uz0, gx, gy, gz);
    const int sgn = side ? -1 : 1;
    T h0 = T(LT::w(0)) * own.A, hout = T(0);  // rest: the node's own equilibrium
    static_for<1, Q>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        const int ck = LT::c(K, axis);
        if (ck == sgn) return;  // unknown: enters from outside
        int sp[3] = {pos[0] - LT::c(K, 0), pos[1] - LT::c(K, 1), pos[2] - LT::c(K, 2)};
        bool inside = true;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (sp[d] < 0 || sp[d] >= n[d]) {
                if (a.periodic[d]) sp[d] = sp[d] < 0 ? sp[d] + n[d] : sp[d] - n[d];
                else inside = false;
            }
        T v;
        bool wall = !inside;
        T ds = T(0), uxs = T(0), uys = T(0), uzs = T(0);
        if (inside) {
            C e0, e1, e2, e3;
            S::load(a.pre, (uint32_t)sp[0] + (uint32_t)a.nx * ((uint32_t)sp[1] + (uint32_t)a.ny * (uint32_t)sp[2]),
                    sc.inv, e0, e1, e2, e3);
            ds = e0;
            uxs = e1;
            uys = e2;
            uzs = e3;
            wall = isnan(ds);
        }
        if (wall) {
            // halfway bounce-back: own previous state in direction inv(K), p(inv K) = -p(K)
            const T p = T(LT::c(K, 0)) * own.Px + T(LT::c(K, 1)) * own.Py + T(LT::c(K, 2)) * own.Pz;
            v = feq_scaled(own.A, own.H, -p);
        } else {
            const NodeMoments<T> m = node_moments<T>(ds, uxs, uys, uzs, gx, gy, gz);
            const T p = T(LT::c(K, 0)) * m.Px + T(LT::c(K, 1)) * m.Py + T(LT::c(K, 2)) * m.Pz;
            v = feq_scaled(m.A, m.H, p);
        }
        v = T(LT::w(K)) * v;
        if (ck == 0) h0 += v;
        else hout += v;
    });
    const T rho_b = T(side ? rho_hi : rho_lo);
    const T drho_b = T((side ? rho_hi : rho_lo) - 1.0);
    const T u = T(sgn) * (drho_b - h0 - T(2) * hout) / rho_b;
    C out[3] = {C(0), C(0), C(0)};
    out[axis] = (C)u;
    step_store<ST>(a.post, i, (C)drho_b, out[0], out[1], out[2], sc.s, a.seed);
}

template <int Q>
cudaError_t launch_q(int storage, const StepArgs& a, int axis, double lo, double hi, cudaStream_t s)
{
    const int n[3] = {a.nx, a.ny, a.nz};
    const int ua = axis == 0 ? 1 : 0, va = axis == 2 ? 1 : 2;
    const int64_t threads = 2 * (int64_t)n[ua] * n[va];
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    switch (storage) {
    case ST_F64: zou_he_kernel<Q, ST_F64><<<blocks, 256, 0, s>>>(a, axis, lo, hi); break;
    case ST_F32: zou_he_kernel<Q, ST_F32><<<blocks, 256, 0, s>>>(a, axis, lo, hi); break;
    case ST_F16S: zou_he_kernel<Q, ST_F16S><<<blocks, 256, 0, s>>>(a, axis, lo, hi); break;
    case ST_BF16S: zou_he_kernel<Q, ST_BF16S><<<blocks, 256, 0, s>>>(a, axis, lo, hi); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_zou_he(int q, int storage, const StepArgs& a, int axis, double rho_lo, double rho_hi,
                          cudaStream_t s)
{
    if (axis < 0 || axis > 2 || a.periodic[axis]) return cudaErrorInvalidValue;
    switch (q) {
    case 9: return launch_q<9>(storage, a, axis, rho_lo, rho_hi, s);
    case 19: return launch_q<19>(storage, a, axis, rho_lo, rho_hi, s);
    case 27: return launch_q<27>(storage, a, axis, rho_lo, rho_hi, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm

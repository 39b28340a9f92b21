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
// state. One thread per face node; a block first evaluates the moments of
// every source node of its 32 x 8 patch of the face once, into shared memory.
// The known populations are evaluated as the step kernels evaluate them, in
// the storage format's compute precision (FP32 for FP32 and 16-bit storage);
// their weighted sums and the face velocity are FP64, because u is the
// difference of two sums of about rho_b - 1 each.
#include "kernels.h"
#include "static_for.cuh"
#include "tau1_node.cuh"

namespace lbm {

namespace {

// Face tile of one block: FU x FV face nodes along the in-face axes, with a
// one-node ring, in the face plane (j = 0) and the plane inside it (j = 1):
// the sources of every known population.
constexpr int FU = 32, FV = 8, SU = FU + 2, SV = FV + 2;

template <typename L> struct FaceMoments {
    L A[2][SV][SU], Px[2][SV][SU], Py[2][SV][SU], Pz[2][SV][SU], H[2][SV][SU];
    unsigned char wall[2][SV][SU];  // outside a non-periodic face, or solid
};

// Box coordinates (x, y, z) of the node at coordinate ca along the face axis
// and (cu, cv) along the in-face axes (the other two, in x, y, z order).
__device__ __forceinline__ uint32_t face_node(const StepArgs& a, int axis, int ca, int cu, int cv)
{
    const int x = axis == 0 ? ca : cu;
    const int y = axis == 0 ? cu : (axis == 1 ? ca : cv);
    const int z = axis == 2 ? ca : cv;
    return (uint32_t)x + (uint32_t)a.nx * ((uint32_t)y + (uint32_t)a.ny * (uint32_t)z);
}

// c (-1 <= c <= n) into [0, n) on a periodic axis; false if c lies outside a
// non-periodic one
__device__ __forceinline__ bool wrap_axis(int& c, int n, bool per)
{
    if (c >= 0 && c < n) return true;
    if (!per) return false;
    c = c < 0 ? c + n : c - n;
    return true;
}

template <int Q, int ST>
__global__ void __launch_bounds__(FU * FV) zou_he_kernel(StepArgs a, int axis, double rho_lo, double rho_hi, int tiles_u,
                                                          int tiles_v)
{
    using S = Storage<ST>;
    using C = typename S::ctype;  // stored values, and the arithmetic of the known populations
    using T = double;             // their sums and the face velocity
    using LT = Lat<Q>;
    __shared__ FaceMoments<C> fm;
    // sizes and periodicity along the face axis and the in-face axes u, v
    const int na = axis == 0 ? a.nx : (axis == 1 ? a.ny : a.nz);
    const int nu = axis == 0 ? a.ny : a.nx;
    const int nv = axis == 2 ? a.ny : a.nz;
    const bool per_u = (axis == 0 ? a.periodic[1] : a.periodic[0]) != 0;
    const bool per_v = (axis == 2 ? a.periodic[1] : a.periodic[2]) != 0;
    int b = blockIdx.x;
    const int side = b / (tiles_u * tiles_v);
    b -= side * tiles_u * tiles_v;
    if (side && na == 1) return;  // one plane: the low face only (the whole block leaves)
    const int u0 = (b % tiles_u) * FU, v0 = (b / tiles_u) * FV;
    const int sgn = side ? -1 : 1;
    const int pa = side ? na - 1 : 0;
    const Scales sc(a.dscale);
    const C gx = gcomp<C>(a, 0), gy = gcomp<C>(a, 1), gz = gcomp<C>(a, 2);

    // every source node's moments, once per block (the face axis is not
    // periodic: the inner plane lies outside only when the box is one plane)
    for (int c = threadIdx.x; c < 2 * SV * SU; c += FU * FV) {
        const int j = c / (SV * SU), r = c - j * (SV * SU), sv = r / SU, su = r - sv * SU;
        const int ca = pa + (j ? sgn : 0);
        int cu = u0 + su - 1, cv = v0 + sv - 1;
        // cells beyond the ring of the face (a patch wider than the face) are
        // the source of no face node: left as walls, never loaded
        const bool near = cu <= nu && cv <= nv;
        const bool inside = near && ca >= 0 && ca < na && wrap_axis(cu, nu, per_u) && wrap_axis(cv, nv, per_v);
        bool wall = !inside;
        NodeMoments<C> m{C(0), C(0), C(0), C(0), C(0)};
        if (inside) {
            C e0, e1, e2, e3;
            S::load(a.pre, face_node(a, axis, ca, cu, cv), sc.inv, e0, e1, e2, e3);
            wall = isnan(e0);
            if (!wall) m = node_moments<C>(e0, e1, e2, e3, gx, gy, gz);
        }
        fm.A[j][sv][su] = m.A;
        fm.Px[j][sv][su] = m.Px;
        fm.Py[j][sv][su] = m.Py;
        fm.Pz[j][sv][su] = m.Pz;
        fm.H[j][sv][su] = m.H;
        fm.wall[j][sv][su] = wall ? 1 : 0;
    }
    __syncthreads();

    const int tu = threadIdx.x % FU, tv = threadIdx.x / FU;
    if (u0 + tu >= nu || v0 + tv >= nv) return;
    if (fm.wall[0][tv + 1][tu + 1]) return;  // solid face node
    const uint32_t i = face_node(a, axis, pa, u0 + tu, v0 + tv);
    NodeMoments<C> own;
    own.A = fm.A[0][tv + 1][tu + 1];
    own.Px = fm.Px[0][tv + 1][tu + 1];
    own.Py = fm.Py[0][tv + 1][tu + 1];
    own.Pz = fm.Pz[0][tv + 1][tu + 1];
    own.H = fm.H[0][tv + 1][tu + 1];
    T h0 = T(LT::w(0)) * T(own.A), hout = T(0);  // rest: the node's own equilibrium
    static_for<1, Q>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int cx = LT::c(K, 0), cy = LT::c(K, 1), cz = LT::c(K, 2);
        const int ck = axis == 0 ? cx : (axis == 1 ? cy : cz);
        if (ck == sgn) return;  // unknown: enters from outside
        // source x - c_K: the face plane (c_K along the axis 0) or the inner plane
        const int j = ck == 0 ? 0 : 1;
        const int su = tu + 1 - (axis == 0 ? cy : cx), sv = tv + 1 - (axis == 2 ? cy : cz);
        C vc;
        if (fm.wall[j][sv][su]) {
            // halfway bounce-back: own previous state in direction inv(K), p(inv K) = -p(K)
            const C p = C(cx) * own.Px + C(cy) * own.Py + C(cz) * own.Pz;
            vc = feq_scaled(own.A, own.H, -p);
        } else {
            const C Px = fm.Px[j][sv][su], Py = fm.Py[j][sv][su], Pz = fm.Pz[j][sv][su];
            const C p = C(cx) * Px + C(cy) * Py + C(cz) * Pz;
            vc = feq_scaled(fm.A[j][sv][su], fm.H[j][sv][su], p);
        }
        const T v = T(LT::w(K)) * T(vc);
        if (ck == 0) h0 += v;
        else hout += v;
    });
    const T rho_b = T(side ? rho_hi : rho_lo);
    const T drho_b = T((side ? rho_hi : rho_lo) - 1.0);
    const T u = T(sgn) * (drho_b - h0 - T(2) * hout) / rho_b;
    const C cu = (C)u;
    step_store<ST>(a.post, i, (C)drho_b, axis == 0 ? cu : C(0), axis == 1 ? cu : C(0), axis == 2 ? cu : C(0), sc.s,
                   a.seed);
}

template <int Q>
cudaError_t launch_q(int storage, const StepArgs& a, int axis, double lo, double hi, cudaStream_t s)
{
    const int nu = axis == 0 ? a.ny : a.nx, nv = axis == 2 ? a.ny : a.nz;  // in-face axes
    const int tu = (nu + FU - 1) / FU, tv = (nv + FV - 1) / FV;
    const int64_t blocks = 2 * (int64_t)tu * tv;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    switch (storage) {
    case ST_F64: zou_he_kernel<Q, ST_F64><<<(unsigned)blocks, FU * FV, 0, s>>>(a, axis, lo, hi, tu, tv); break;
    case ST_F32: zou_he_kernel<Q, ST_F32><<<(unsigned)blocks, FU * FV, 0, s>>>(a, axis, lo, hi, tu, tv); break;
    case ST_F16S: zou_he_kernel<Q, ST_F16S><<<(unsigned)blocks, FU * FV, 0, s>>>(a, axis, lo, hi, tu, tv); break;
    case ST_BF16S: zou_he_kernel<Q, ST_BF16S><<<(unsigned)blocks, FU * FV, 0, s>>>(a, axis, lo, hi, tu, tv); break;
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

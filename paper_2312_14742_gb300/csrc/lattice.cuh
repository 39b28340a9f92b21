// Lattice tables of the CUDA path (D3Q19, D3Q27), typed for this library.
//
// Order: rest; the 6 faces; the 12 edges; the 8 corners. Each direction is
// followed by its opposite, so inv(k) = k + 1 for odd k and k - 1 for even k.
// Weights are the textbook ones for c_s^2 = 1/3 (Qian et al. 1992), by
// class: D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216.
#pragma once

namespace lbm {

// Velocity component a (0 = x, 1 = y, 2 = z) of direction k.
__host__ __device__ constexpr int cvel(int k, int a)
{
    constexpr int T[27][3] = {
        { 0, 0, 0},
        { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1},
        { 1, 1, 0}, {-1,-1, 0}, { 1,-1, 0}, {-1, 1, 0}, { 1, 0, 1}, {-1, 0,-1},
        { 1, 0,-1}, {-1, 0, 1}, { 0, 1, 1}, { 0,-1,-1}, { 0, 1,-1}, { 0,-1, 1},
        { 1, 1, 1}, {-1,-1,-1}, { 1, 1,-1}, {-1,-1, 1}, { 1,-1, 1}, {-1, 1,-1},
        {-1, 1, 1}, { 1,-1,-1}};
    return T[k][a];
}

__host__ __device__ constexpr int inv_dir(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }

// 0 rest, 1 face, 2 edge, 3 corner: the squared speed |c_k|^2.
__host__ __device__ constexpr int dir_class(int k) { return k == 0 ? 0 : (k < 7 ? 1 : (k < 19 ? 2 : 3)); }

template <int Q> struct Weights;
template <> struct Weights<19> {
    static constexpr int NCLASS = 3;
    __host__ __device__ static constexpr double w(int cls)
    {
        return cls == 0 ? 1.0 / 3.0 : (cls == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};
template <> struct Weights<27> {
    static constexpr int NCLASS = 4;
    __host__ __device__ static constexpr double w(int cls)
    {
        return cls == 0 ? 8.0 / 27.0 : (cls == 1 ? 2.0 / 27.0 : (cls == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
};

}  // namespace lbm

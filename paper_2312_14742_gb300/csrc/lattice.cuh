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

// D2Q9 (one plane): rest; (+1,0), (-1,0), (0,+1), (0,-1); (+1,+1), (-1,-1),
// (+1,-1), (-1,+1). inv(k) = k + 1 for odd k, k - 1 for even k. Weights by
// class (rest, axis, diagonal): 4/9, 1/9, 1/36.
__host__ __device__ constexpr int c2(int k, int a)
{
    constexpr int T[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    return a < 2 ? T[k][a] : 0;
}
__host__ __device__ constexpr int inv2(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }
__host__ __device__ constexpr int class2(int k) { return k == 0 ? 0 : (k < 5 ? 1 : 2); }
__host__ __device__ constexpr double w2(int cls) { return cls == 0 ? 4.0 / 9.0 : (cls == 1 ? 1.0 / 9.0 : 1.0 / 36.0); }

// One interface to the three lattices: velocity component, opposite, weight.
template <int Q> struct Lat {
    __host__ __device__ static constexpr int c(int k, int a) { return cvel(k, a); }
    __host__ __device__ static constexpr int inv(int k) { return inv_dir(k); }
    __host__ __device__ static constexpr double w(int k) { return Weights<Q>::w(dir_class(k)); }
};
template <> struct Lat<9> {
    __host__ __device__ static constexpr int c(int k, int a) { return c2(k, a); }
    __host__ __device__ static constexpr int inv(int k) { return inv2(k); }
    __host__ __device__ static constexpr double w(int k) { return w2(class2(k)); }
};

}  // namespace lbm

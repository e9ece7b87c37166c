// Lattice velocity sets and weights for the GPU path.
//
// D2Q9 follows the ordering printed in Appendix A of the paper:
//   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
// with w = 4/9, 1/9 (axes), 1/36 (diagonals).
// D3Q19 (the 3D extension) uses rest, the six axis directions in +/- pairs,
// then the twelve edge diagonals in +/- pairs:
//   1 +x 2 -x 3 +y 4 -y 5 +z 6 -z
//   7 (+x+y) 8 (-x-y) 9 (+x-y) 10 (-x+y) 11 (+x+z) 12 (-x-z) 13 (+x-z) 14 (-x+z)
//   15 (+y+z) 16 (-y-z) 17 (+y-z) 18 (-y+z)
// with w = 1/3, 1/18 (axes), 1/36 (edges).  Populations cross the C ABI in
// these orders.
#pragma once

#include <cstdint>

namespace lbmgpu {

template <int Q> struct Lattice;

template <> struct Lattice<9> {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        return i == 1 ? 1 : i == 3 ? -1 : (i == 5 || i == 8) ? 1 : (i == 6 || i == 7) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int i) {
        return i == 2 ? 1 : i == 4 ? -1 : (i == 5 || i == 6) ? 1 : (i == 7 || i == 8) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <> struct Lattice<19> {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    // +/- pairs: direction 2k-1 and 2k are opposite
    __host__ __device__ static constexpr int sgn(int i) { return (i & 1) ? 1 : -1; }
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 2) ? sgn(i)
             : (i >= 7 && i <= 10) ? ((i == 7 || i == 9) ? 1 : -1)
             : (i >= 11 && i <= 14) ? ((i == 11 || i == 13) ? 1 : -1) : 0;
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 3 || i == 4) ? sgn(i)
             : (i >= 7 && i <= 10) ? ((i == 7 || i == 10) ? 1 : -1)
             : (i >= 15 && i <= 18) ? ((i == 15 || i == 17) ? 1 : -1) : 0;
    }
    __host__ __device__ static constexpr int cz(int i) {
        return (i == 5 || i == 6) ? sgn(i)
             : (i >= 11 && i <= 14) ? ((i == 11 || i == 14) ? 1 : -1)
             : (i >= 15 && i <= 18) ? ((i == 15 || i == 18) ? 1 : -1) : 0;
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

}  // namespace lbmgpu
